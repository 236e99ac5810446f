"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle (never the CUDA path) against something other than
itself: printed closed forms, printed tables, textbook identities, brute force.
"""
import itertools
import math

import numpy as np
import pytest

from conftest import load_golden

CS2 = 1.0 / 3.0


def K(a, b, c):
    return a + 3 * b + 9 * c


def rand_state(rng):
    rho = rng.uniform(0.5, 2.0)
    p = rng.uniform(0.01, 0.6)
    u = rng.uniform(-1.0, 1.0, 3)
    u *= rng.uniform(0.0, 0.1) / max(np.linalg.norm(u), 1e-12)
    return rho, p, u


# ---- lattice (Sec. II.A) ----------------------------------------------------

def test_velocity_table_matches_printed_matrix(orc):
    rows = load_golden("d3q27_velocities.txt")
    printed = np.array([[int(v) for v in r] for r in rows]).T  # [27, 3]
    c, w = orc.lattice()
    assert np.array_equal(c, printed)
    # opposite of every odd i is i + 1 (used by bounce-back)
    for i in range(1, 27, 2):
        assert np.array_equal(c[i], -c[i + 1])


def test_weights_isotropy(orc):
    """Weights of Sec. II.A: normalisation and isotropy up to 4th order."""
    c, w = orc.lattice()
    cf = c.astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ cf, 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, cf, cf), CS2 * np.eye(3), atol=1e-16)
    # sum w c_a c_b c_c c_d = cs^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
    T = np.einsum("i,ia,ib,ic,id->abcd", w, cf, cf, cf, cf)
    d = np.eye(3)
    ref = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(T, ref, atol=1e-16)


def test_hermite_orthogonality(orc):
    """App. B polynomials are orthogonal under the weights with norm a!b!c! cs2^(a+b+c)."""
    c, w = orc.lattice()
    orders = list(itertools.product(range(3), repeat=3))
    H = np.array([[orc.hermite(i, *o) for o in orders] for i in range(27)])
    G = H.T @ (w[:, None] * H)
    norm = np.array([math.factorial(a) * math.factorial(b) * math.factorial(cc) * CS2 ** (a + b + cc)
                     for (a, b, cc) in orders])
    assert np.allclose(G, np.diag(norm), atol=1e-15)
    # second-order Hermite polynomial spot values: H_{i200} = c_ix^2 - cs^2
    assert abs(orc.hermite(1, 2, 0, 0) - (1 - CS2)) < 1e-16
    assert abs(orc.hermite(3, 2, 0, 0) - (0 - CS2)) < 1e-16


# ---- equilibria (Sec. III) ----------------------------------------------------

def closed_form_keq(model, rho, p, u):
    """Equilibrium central moments as printed in Secs. III.A-III.D."""
    ux, uy, uz = u
    d = p - rho * CS2
    cs4 = CS2 * CS2
    k = np.zeros(27)
    k[K(0, 0, 0)] = rho
    k[K(2, 0, 0)] = k[K(0, 2, 0)] = k[K(0, 0, 2)] = p
    if model == "A":
        k[K(1, 2, 0)] = -d * ux - rho * ux * uy ** 2
        k[K(1, 0, 2)] = -d * ux - rho * ux * uz ** 2
        k[K(0, 1, 2)] = -d * uy - rho * uy * uz ** 2
        k[K(2, 1, 0)] = -d * uy - rho * ux ** 2 * uy
        k[K(2, 0, 1)] = -d * uz - rho * ux ** 2 * uz
        k[K(0, 2, 1)] = -d * uz - rho * uy ** 2 * uz
        k[K(1, 1, 1)] = -rho * ux * uy * uz
        k[K(2, 2, 0)] = p * CS2 + d * (ux ** 2 + uy ** 2) + 3 * rho * ux ** 2 * uy ** 2
        k[K(2, 0, 2)] = p * CS2 + d * (ux ** 2 + uz ** 2) + 3 * rho * ux ** 2 * uz ** 2
        k[K(0, 2, 2)] = p * CS2 + d * (uy ** 2 + uz ** 2) + 3 * rho * uy ** 2 * uz ** 2
        k[K(2, 1, 1)] = d * uy * uz + 3 * rho * ux ** 2 * uy * uz
        k[K(1, 2, 1)] = d * ux * uz + 3 * rho * ux * uy ** 2 * uz
        k[K(1, 1, 2)] = d * ux * uy + 3 * rho * ux * uy * uz ** 2
        k[K(1, 2, 2)] = -d * ux * (uy ** 2 + uz ** 2 + CS2) - rho * ux * (6 * uy ** 2 * uz ** 2 + CS2 * (uy ** 2 + uz ** 2))
        k[K(2, 1, 2)] = -d * uy * (ux ** 2 + uz ** 2 + CS2) - rho * uy * (6 * ux ** 2 * uz ** 2 + CS2 * (ux ** 2 + uz ** 2))
        k[K(2, 2, 1)] = -d * uz * (ux ** 2 + uy ** 2 + CS2) - rho * uz * (6 * ux ** 2 * uy ** 2 + CS2 * (ux ** 2 + uy ** 2))
        k[K(2, 2, 2)] = (p * cs4 + d * (ux ** 2 * uy ** 2 + ux ** 2 * uz ** 2 + uy ** 2 * uz ** 2
                                        + CS2 * (ux ** 2 + uy ** 2 + uz ** 2))
                         + rho * (10 * ux ** 2 * uy ** 2 * uz ** 2
                                  + 3 * CS2 * (ux ** 2 * uy ** 2 + ux ** 2 * uz ** 2 + uy ** 2 * uz ** 2)))
    elif model == "B":
        k[K(1, 2, 0)] = k[K(1, 0, 2)] = -d * ux
        k[K(0, 1, 2)] = k[K(2, 1, 0)] = -d * uy
        k[K(2, 0, 1)] = k[K(0, 2, 1)] = -d * uz
        k[K(2, 2, 0)] = p * CS2 + d * (ux ** 2 + uy ** 2)
        k[K(2, 0, 2)] = p * CS2 + d * (ux ** 2 + uz ** 2)
        k[K(0, 2, 2)] = p * CS2 + d * (uy ** 2 + uz ** 2)
        k[K(2, 1, 1)] = d * uy * uz
        k[K(1, 2, 1)] = d * ux * uz
        k[K(1, 1, 2)] = d * ux * uy
        k[K(1, 2, 2)] = -d * ux * (uy ** 2 + uz ** 2 + CS2)
        k[K(2, 1, 2)] = -d * uy * (ux ** 2 + uz ** 2 + CS2)
        k[K(2, 2, 1)] = -d * uz * (ux ** 2 + uy ** 2 + CS2)
        k[K(2, 2, 2)] = p * cs4 + d * (ux ** 2 * uy ** 2 + ux ** 2 * uz ** 2 + uy ** 2 * uz ** 2
                                       + CS2 * (ux ** 2 + uy ** 2 + uz ** 2))
    elif model == "C":
        k[K(2, 2, 0)] = p * CS2 - d * (ux ** 2 + uy ** 2)
        k[K(2, 0, 2)] = p * CS2 - d * (ux ** 2 + uz ** 2)
        k[K(0, 2, 2)] = p * CS2 - d * (uy ** 2 + uz ** 2)
        k[K(2, 1, 1)] = -d * uy * uz
        k[K(1, 2, 1)] = -d * ux * uz
        k[K(1, 1, 2)] = -d * ux * uy
        k[K(1, 2, 2)] = d * ux * (2 * uy ** 2 + 2 * uz ** 2 + CS2)
        k[K(2, 1, 2)] = d * uy * (2 * ux ** 2 + 2 * uz ** 2 + CS2)
        k[K(2, 2, 1)] = d * uz * (2 * ux ** 2 + 2 * uy ** 2 + CS2)
        k[K(2, 2, 2)] = p * cs4 - 3 * d * (ux ** 2 * uy ** 2 + ux ** 2 * uz ** 2 + uy ** 2 * uz ** 2
                                           + CS2 * (ux ** 2 + uy ** 2 + uz ** 2))
    elif model == "D":
        k[K(2, 2, 0)] = k[K(2, 0, 2)] = k[K(0, 2, 2)] = p * CS2
        k[K(2, 2, 2)] = p * cs4
    return k


@pytest.mark.parametrize("model,code", [("A", 0), ("B", 1), ("C", 2), ("D", 3)])
def test_equilibrium_central_moments_match_printed_closed_forms(orc, model, code):
    """P1: Hermite f^eq -> central moments by definition == printed closed forms."""
    rng = np.random.default_rng(11 + code)
    worst = 0.0
    for _ in range(2000):
        rho, p, u = rand_state(rng)
        k = orc.central_moments(orc.feq(code, rho, p, u), u)
        ref = closed_form_keq(model, rho, p, u)
        worst = max(worst, np.abs(k - ref).max() / rho)
    assert worst < 5e-15, worst


def test_standard_and_li_forms_equal_general_form(orc):
    """Eq. (standard CG 2nd) == g2 + (p - rho cs2) E_i, and Li et al.'s original
    == g2 + (p - rho cs2)(E_i + Phi_i^(3)) (Secs. III, III.C)."""
    rng = np.random.default_rng(5)
    for _ in range(500):
        rho, p, u = rand_state(rng)
        assert np.allclose(orc.feq(0, rho, p, u), orc.feq(5, rho, p, u), atol=2e-15, rtol=0)
        assert np.allclose(orc.feq(4, rho, p, u), orc.feq(6, rho, p, u), atol=2e-15, rtol=0)


def test_third_order_moments_of_generalized_equilibria(orc):
    """P2: third-order raw moments of Model D f^eq (Sec. III.E)."""
    c, w = orc.lattice()
    cf = c.astype(float)
    rng = np.random.default_rng(7)
    for _ in range(300):
        rho, p, u = rand_state(rng)
        f = orc.feq(3, rho, p, u)
        T = np.einsum("i,ia,ib,ic->abc", f, cf, cf, cf)
        d = np.eye(3)
        for a, b, cc in itertools.product(range(3), repeat=3):
            iso = u[a] * d[b, cc] + u[b] * d[a, cc] + u[cc] * d[a, b]
            if a == b == cc:
                ref = rho * CS2 * iso
            else:
                ref = p * iso + rho * u[a] * u[b] * u[cc]
            assert abs(T[a, b, cc] - ref) < 1e-15 * max(1.0, rho)


def test_low_order_moments_of_equilibria(orc):
    """Mass, momentum and the Navier-Stokes stress p I + rho u u for all models."""
    c, w = orc.lattice()
    cf = c.astype(float)
    rng = np.random.default_rng(8)
    for model in range(4):
        for _ in range(100):
            rho, p, u = rand_state(rng)
            f = orc.feq(model, rho, p, u)
            assert abs(f.sum() - rho) < 1e-15
            assert np.allclose(f @ cf, rho * u, atol=1e-16)
            S = np.einsum("i,ia,ib->ab", f, cf, cf)
            assert np.allclose(S, p * np.eye(3) + rho * np.outer(u, u), atol=1e-15)


# ---- moment transforms (Sec. II.B) ---------------------------------------------

def test_moment_matrix_inverse(orc):
    """P3: M M^-1 = I and M^-1 equals the tensor product of the textbook 1D
    three-point inverse f(-1)=(m2-m1)/2, f(0)=m0-m2, f(1)=(m1+m2)/2."""
    M = orc.moment_matrix()
    Minv = orc.moment_matrix_inverse()
    assert np.abs(M @ Minv - np.eye(27)).max() < 1e-14
    assert np.abs(Minv @ M - np.eye(27)).max() < 1e-14
    inv1 = {-1: [0.0, -0.5, 0.5], 0: [1.0, 0.0, -1.0], 1: [0.0, 0.5, 0.5]}
    c, _ = orc.lattice()
    ref = np.zeros((27, 27))
    for i in range(27):
        for a, b, cc in itertools.product(range(3), repeat=3):
            ref[i, K(a, b, cc)] = inv1[c[i, 0]][a] * inv1[c[i, 1]][b] * inv1[c[i, 2]][cc]
    assert np.abs(Minv - ref).max() < 1e-15


def test_raw_moments_are_matrix_product(orc):
    rng = np.random.default_rng(2)
    f = rng.uniform(0, 1, 27)
    assert np.allclose(orc.raw_moments(f), orc.moment_matrix() @ f, atol=1e-15)


def test_central_moment_roundtrip_and_brute_force(orc):
    """k by definition, then binomial shift + M^-1 returns f; k also equals the
    brute-force sum over (c - u) powers computed here."""
    c, w = orc.lattice()
    rng = np.random.default_rng(3)
    for _ in range(200):
        f = w * (1.0 + 0.2 * rng.standard_normal(27))
        u = rng.uniform(-0.2, 0.2, 3)
        k = orc.central_moments(f, u)
        ref = np.array([sum(f[i] * (c[i, 0] - u[0]) ** a * (c[i, 1] - u[1]) ** b * (c[i, 2] - u[2]) ** cc
                            for i in range(27))
                        for cc in range(3) for b in range(3) for a in range(3)])
        assert np.abs(k - ref).max() < 1e-15
        assert np.abs(orc.cm_to_f(k, u) - f).max() < 1e-15


# ---- collision (Sec. II.B and III.E) -------------------------------------------

def test_equal_rates_collision_is_bgk(orc):
    """P7: all relaxation rates equal, no force, no Q -> lattice BGK toward the
    Model D equilibrium (Eq. collision_bgk), through the full 27-moment transform."""
    c, w = orc.lattice()
    rng = np.random.default_rng(4)
    for _ in range(200):
        _, p, u = rand_state(rng)
        f = w * rng.uniform(0.5, 2.0) * (1.0 + 0.1 * rng.standard_normal(27))
        rho = f.sum()
        om = rng.uniform(0.2, 1.9)
        feq = orc.feq(3, rho, p, u)
        k = orc.central_moments(f, u)
        keq = orc.central_moments(feq, u)
        ks = orc.collide_cm(k, keq, np.full(11, om), np.zeros(3), np.zeros(3))
        fs = orc.cm_to_f(ks, u)
        assert np.abs(fs - (f - om * (f - feq))).max() < 2e-15


def test_collision_matches_printed_unit_rate_form(orc):
    """All rates 1 except omega_1: the general form reduces to the printed
    Eq. (collision_step_with_all_one) and the concise Model D form."""
    rng = np.random.default_rng(6)
    for _ in range(300):
        rho, p, u = rand_state(rng)
        k = rng.standard_normal(27) * 0.1
        k[0] = rho
        F = rng.standard_normal(3) * 1e-3
        Q = rng.standard_normal(3) * 1e-3
        om1 = rng.uniform(0.1, 1.95)
        om = np.ones(11); om[1] = om1
        keq = closed_form_keq("D", rho, p, u)
        ks = orc.collide_cm(k, keq, om, F, Q)
        cs4 = CS2 ** 2
        ref = {
            (1, 0, 0): F[0] / 2, (0, 1, 0): F[1] / 2, (0, 0, 1): F[2] / 2,
            (1, 1, 0): (1 - om1) * k[K(1, 1, 0)], (0, 1, 1): (1 - om1) * k[K(0, 1, 1)],
            (1, 0, 1): (1 - om1) * k[K(1, 0, 1)],
            (1, 2, 0): CS2 * F[0] / 2, (1, 0, 2): CS2 * F[0] / 2,
            (2, 1, 0): CS2 * F[1] / 2, (0, 1, 2): CS2 * F[1] / 2,
            (2, 0, 1): CS2 * F[2] / 2, (0, 2, 1): CS2 * F[2] / 2, (1, 1, 1): 0.0,
            (2, 2, 0): p * CS2, (2, 0, 2): p * CS2, (0, 2, 2): p * CS2,
            (2, 1, 1): 0.0, (1, 2, 1): 0.0, (1, 1, 2): 0.0,
            (1, 2, 2): cs4 * F[0] / 2, (2, 1, 2): cs4 * F[1] / 2, (2, 2, 1): cs4 * F[2] / 2,
            (2, 2, 2): p * cs4,
        }
        for (a, b, cc), v in ref.items():
            assert abs(ks[K(a, b, cc)] - v) < 1e-15, (a, b, cc)
        d1 = (1 - om1) * (k[K(2, 0, 0)] - k[K(0, 2, 0)]) + (1 - om1 / 2) * (Q[0] - Q[1])
        d2 = (1 - om1) * (k[K(2, 0, 0)] - k[K(0, 0, 2)]) + (1 - om1 / 2) * (Q[0] - Q[2])
        tr = 3 * p + Q.sum() / 2
        assert abs(ks[K(2, 0, 0)] - ks[K(0, 2, 0)] - d1) < 1e-15
        assert abs(ks[K(2, 0, 0)] - ks[K(0, 0, 2)] - d2) < 1e-15
        assert abs(ks[K(2, 0, 0)] + ks[K(0, 2, 0)] + ks[K(0, 0, 2)] - tr) < 2e-15
        assert ks[0] == k[0]


def test_first_order_moment_after_collision_is_half_force(orc):
    """P5: with u including F/2, k100 = -F_x/2, so k100* = F_x/2 for any omega_0."""
    rng = np.random.default_rng(9)
    c, w = orc.lattice()
    for _ in range(100):
        f = w * (1 + 0.1 * rng.standard_normal(27))
        F = rng.standard_normal(3) * 1e-2
        rho = f.sum()
        u = (f @ c.astype(float) + F / 2) / rho
        k = orc.central_moments(f, u)
        assert np.allclose(k[[K(1, 0, 0), K(0, 1, 0), K(0, 0, 1)]], -F / 2, atol=1e-16)
        om = rng.uniform(0.1, 1.9, 11)
        ks = orc.collide_cm(k, np.zeros(27), om, F, np.zeros(3))
        assert np.allclose(ks[[K(1, 0, 0), K(0, 1, 0), K(0, 0, 1)]], F / 2, atol=1e-16)


# ---- equation of state (Sec. II.A) against printed Mach numbers -------------------

def test_eos_against_printed_bubble_mach_numbers(orc):
    """(c_s^k)^2 = xi (1 - alpha_k) with the lighter phase at alpha = 8/27 gives
    the printed liquid Mach numbers of the rising-bubble cases (Sec. IV.D)."""
    from paper_2309_07801_gb300.inputs import rest_fractions
    for row in load_golden("bubble_mach.txt"):
        _, rr0, rb0, g, nx, ma = row
        rr0, rb0, g, nx, ma = float(rr0), float(rb0), float(g), int(nx), float(ma)
        ar, ab = rest_fractions(rr0, rb0)
        assert abs(ab - 8 / 27) < 1e-15
        # a pure red (liquid) cell at rest: p / rho_r = (c_s^r)^2 from the oracle's EOS
        P = orc.make_params(1, 1, 1, rho_r0=rr0, rho_b0=rb0, alpha_r=ar, alpha_b=ab)
        d = orc.Domain(P)
        d.init(np.full((1, 1, 1), rr0), np.zeros((1, 1, 1)), np.zeros((3, 1, 1, 1)))
        cs_r = math.sqrt(d.macros()["p"].item() / rr0)
        U = math.sqrt(g * nx / 2)
        assert abs(U / cs_r - ma) / ma < 0.005, (U / cs_r, ma)


def test_layered_table_rest_fractions_are_consistent():
    """The printed alpha_b of the layered-flow cases satisfy the pressure balance
    gamma = (1-alpha_b)/(1-alpha_r) with alpha_r in (0, 1) (Sec. II.A reading)."""
    for row in load_golden("layered_table.txt"):
        _, rr0, rb0, ab, M = row
        gamma = float(rr0) / float(rb0)
        ar = 1 - (1 - float(ab)) / gamma
        assert 0.0 < ar < 1.0
