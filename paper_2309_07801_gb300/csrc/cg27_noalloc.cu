// cg27_noalloc.cu -- per-colour mass reduction that allocates nothing.
//
// cg_mass_noalloc() sums two density fields in FP64, in a fixed order, with its
// block partial sums kept in a file-scope __device__ array instead of a
// caller-supplied workspace.  It exists for callers that cannot allocate device
// memory at the point where they need the sums: code that only holds device
// pointers to density fields and owns no domain workspace, or code running
// where a cudaMalloc is not allowed (it may synchronise the whole device, or
// all device memory is already reserved by another allocator).  The array is
// 64 KiB and every GPU that loads this library holds it until the process
// exits.
#include "cg27.h"

#include <cuda_runtime.h>

#include <mutex>
#include <string>

namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_CELLS_PER_BLOCK = 16384;  // 64 cells per thread
constexpr int NA_MAX_BLOCKS = CG_NOALLOC_MAX_CELLS / NA_CELLS_PER_BLOCK;
static_assert((long long)NA_MAX_BLOCKS * NA_CELLS_PER_BLOCK == CG_NOALLOC_MAX_CELLS,
              "the cell limit must be a whole number of blocks");

// block partial sums (red, blue) followed by the two totals
static __device__ __align__(256) double g_noalloc_scratch[2 * NA_MAX_BLOCKS + 2];

// device address of g_noalloc_scratch, looked up once per device
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

}  // namespace

// records the message returned by cg_last_error() (defined in cg27_capi.cu)
int cg27_internal_fail(int code, const char* msg);

namespace {

int na_fail(int code, const std::string& msg) { return cg27_internal_fail(code, msg.c_str()); }

template <typename T>
__global__ void __launch_bounds__(NA_THREADS)
k_mass_partial_noalloc(const T* rho_r, const T* rho_b, long long n, double* partial) {
  __shared__ double sr[NA_THREADS], sb[NA_THREADS];
  const long long lo = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
  const long long hi = (lo + NA_CELLS_PER_BLOCK < n) ? lo + NA_CELLS_PER_BLOCK : n;
  double ar = 0.0, ab = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += NA_THREADS) {
    ar += double(rho_r[i]);
    ab += double(rho_b[i]);
  }
  sr[threadIdx.x] = ar;
  sb[threadIdx.x] = ab;
  __syncthreads();
  for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sr[0];
    partial[2 * blockIdx.x + 1] = sb[0];
  }
}

// sums the first nblocks partials in a fixed order; writes both totals
__global__ void __launch_bounds__(NA_THREADS)
k_mass_final_noalloc(const double* partial, int nblocks, double* out) {
  __shared__ double sr[NA_THREADS], sb[NA_THREADS];
  double ar = 0.0, ab = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += NA_THREADS) {
    ar += partial[2 * i];
    ab += partial[2 * i + 1];
  }
  sr[threadIdx.x] = ar;
  sb[threadIdx.x] = ab;
  __syncthreads();
  for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sr[0];
    out[1] = sb[0];
  }
}

// device address of the scratch array on the current device (set-up on first use)
int scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(CG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(CG_ERR_UNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(CG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return CG_OK;
}

}  // namespace

extern "C" int cg_mass_noalloc(const void* d_rho_r, const void* d_rho_b, int64_t n, int32_t precision,
                               void* cuda_stream, double out_mass[2]) {
  if (!out_mass) return na_fail(CG_ERR_INVALID_ARG, "out_mass is NULL");
  if (n < 0) return na_fail(CG_ERR_INVALID_ARG, "n must be >= 0");
  if (n > CG_NOALLOC_MAX_CELLS)
    return na_fail(CG_ERR_INVALID_ARG, "n = " + std::to_string(n) + " exceeds the " +
                                           std::to_string((long long)CG_NOALLOC_MAX_CELLS) +
                                           "-cell limit of the static scratch; use cg_reduce()");
  if (precision != CG_F64 && precision != CG_F32)
    return na_fail(CG_ERR_INVALID_ARG, "precision must be CG_F64 or CG_F32");
  if (n > 0 && (!d_rho_r || !d_rho_b)) return na_fail(CG_ERR_INVALID_ARG, "density pointer is NULL");
  if (n == 0) {
    out_mass[0] = out_mass[1] = 0.0;
    return CG_OK;
  }
  double* scratch = nullptr;
  int rc = scratch_on_current_device(&scratch);
  if (rc != CG_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nblocks = (int)((n + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
  double* partial = scratch;
  double* total = scratch + 2 * NA_MAX_BLOCKS;
  if (precision == CG_F64)
    k_mass_partial_noalloc<double><<<nblocks, NA_THREADS, 0, st>>>(
        static_cast<const double*>(d_rho_r), static_cast<const double*>(d_rho_b), n, partial);
  else
    k_mass_partial_noalloc<float><<<nblocks, NA_THREADS, 0, st>>>(
        static_cast<const float*>(d_rho_r), static_cast<const float*>(d_rho_b), n, partial);
  k_mass_final_noalloc<<<1, NA_THREADS, 0, st>>>(partial, nblocks, total);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(CG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  double host[2];
  e = cudaMemcpyAsync(host, total, sizeof(host), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(CG_ERR_CUDA, std::string("read-back: ") + cudaGetErrorString(e));
  out_mass[0] = host[0];
  out_mass[1] = host[1];
  return CG_OK;
}
