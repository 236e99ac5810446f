"""The dependency edges of the slab-pipeline step graphs order every pair of
conflicting memory accesses (no GPU).

A model of the step on a column of nz planes (the x-y extent does not matter
for z slabs): each graph node (pass of one slab in one step) gets the set of
locations it reads and writes, with the plane halos and prefetches of the
kernels in cg27_step.cuh:
  macro   reads  F pulled (planes z-1..z+1), fractions of S_in on [zb-1, ze+1],
                 DIVR and REST of S_in on the slab; writes MAC, PHI
  fields  reads  PHI on [zb-2, ze+2], MAC on [zb, ze];
          writes FORCE, WV, fractions, R and REST of S_out
  div     reads  WV and R of S_out on [zb-1, ze]; writes QC, DIVR of S_out
  collide reads  F pulled, MAC on [zb-1, ze] (walls), FORCE, QC, REST of S_in
                 and S_out on the slab; writes F
Populations are modelled per slot (direction, plane) with the directions
c_z in {-1, 0, 1}: with two buffers a step pulls (q, z - c_q) from buffer
parity and writes (q, z) of the other; in place, even steps read (q, z) and
write (opp q, z), odd steps read (opp q, z - c_q) and write (q, z + c_q).
The graph's edges are those the library builds: fields(i) after
macro(i-1..i+1), div(i) after fields(i-1..i+1), collide(i) after div(i), and
macro(t+1, i) after collide(t, i-1..i+1).  Every pair of nodes that touch a
location, one of them writing, must be ordered by a path in the graph, in the
order of the sequential step (and two slabs of one pass must not conflict).

The fused form (FP32, two buffers) has three passes per slab: fields, div and
  fused   reads  F pulled and mac[t & 1], FORCE, QC and the fractions of S_out
                 on the source planes [zb-1, ze] (the tile's planes plus one
                 recomputed plane on either side), DIVR of S_out on the slab;
                 writes F, mac[(t+1) & 1] and PHI on the slab
(fields then reads mac[t & 1]), with the edges fields(t, i) after fused(t-1,
i-1..i+1), div(i) after fields(i-1..i+1), fused(i) after div(i-1..i+1).
"""
import itertools

import pytest

PASSES = ("macro", "fields", "div", "collide")


def _slabs(nz, planes):
    ns = (nz + planes - 1) // planes
    return [(i * planes, min(nz, (i + 1) * planes)) for i in range(ns)]


def _pop_slots(nz, zb, ze, mode, step):
    """(reads, writes) of the populations by the cells of planes [zb, ze)."""
    rd, wr = set(), set()
    for z in range(zb, ze):
        for q in range(3):
            c = q - 1
            opp = 2 - q
            if mode == "two_buffers":
                par = step & 1
                rd.add(("F%d" % par, q, (z - c) % nz))
                wr.add(("F%d" % (1 - par), q, z))
            elif step % 2 == 0:  # in place, even step
                rd.add(("F", q, z))
                wr.add(("F", opp, z))
            else:  # in place, odd step
                rd.add(("F", opp, (z - c) % nz))
                wr.add(("F", q, (z + c) % nz))
    return rd, wr


def _planes(field, lo, hi, nz):
    return {(field, z % nz) for z in range(lo, hi + 1)}


def _accesses(nz, zb, ze, pass_, mode, step):
    s_in, s_out = "S%d" % (step & 1), "S%d" % (1 - (step & 1))
    last = ze - 1
    if pass_ == "macro":
        pr, _ = _pop_slots(nz, zb, ze, mode, step)
        rd = pr | _planes(s_in + ".frac", zb - 1, ze + 1, nz) | _planes(s_in + ".divr", zb, last, nz) \
            | _planes(s_in + ".rest", zb, last, nz)
        wr = _planes("mac", zb, last, nz) | _planes("phi", zb, last, nz)
    elif pass_ == "fields":
        rd = _planes("phi", zb - 2, ze + 2, nz) | _planes("mac", zb, ze, nz)
        wr = set()
        for f in ("force", "wv", s_out + ".frac", s_out + ".R", s_out + ".rest"):
            wr |= _planes(f, zb, last, nz)
    elif pass_ == "div":
        rd = _planes("wv", zb - 1, ze, nz) | _planes(s_out + ".R", zb - 1, ze, nz)
        wr = _planes("qc", zb, last, nz) | _planes(s_out + ".divr", zb, last, nz)
    else:
        pr, pw = _pop_slots(nz, zb, ze, mode, step)
        rd = pr | _planes("mac", zb - 1, ze, nz)
        for f in ("force", "qc", s_in + ".rest", s_out + ".rest"):
            rd |= _planes(f, zb, last, nz)
        wr = pw
    return rd, wr


def _fused_accesses(nz, zb, ze, pass_, step):
    s_out = "S%d" % (1 - (step & 1))
    mac, mac_next = "mac%d" % (step & 1), "mac%d" % (1 - (step & 1))
    last = ze - 1
    if pass_ == "fields":
        rd = _planes("phi", zb - 2, ze + 2, nz) | _planes(mac, zb, ze, nz)
        wr = set()
        for f in ("force", "wv", s_out + ".frac", s_out + ".R"):
            wr |= _planes(f, zb, last, nz)
    elif pass_ == "div":
        rd = _planes("wv", zb - 1, ze, nz) | _planes(s_out + ".R", zb - 1, ze, nz)
        wr = _planes("qc", zb, last, nz) | _planes(s_out + ".divr", zb, last, nz)
    else:
        pr, _ = _pop_slots(nz, zb - 1, ze + 1, "two_buffers", step)
        _, pw = _pop_slots(nz, zb, ze, "two_buffers", step)
        rd = pr | _planes(s_out + ".divr", zb, last, nz)
        for f in (mac, "force", "qc", s_out + ".frac"):
            rd |= _planes(f, zb - 1, ze, nz)
        wr = pw | _planes(mac_next, zb, last, nz) | _planes("phi", zb, last, nz)
    return rd, wr


def _fused_graph(ns, nsteps, fused_pred=None):
    pred = {}
    near = lambda i: {(i + d) % ns for d in (-1, 0, 1)}
    for t in range(nsteps):
        for i in range(ns):
            pred[(t, 0, i)] = {(t - 1, 2, j) for j in near(i)} if t > 0 else set()
            pred[(t, 1, i)] = {(t, 0, j) for j in near(i)}
            pred[(t, 2, i)] = {(t, 1, j) for j in (near(i) if fused_pred is None else fused_pred(i))}
    return pred


def _unordered(acc, anc):
    bad = []
    for u, v in itertools.combinations(sorted(acc), 2):
        (ru, wu), (rv, wv) = acc[u], acc[v]
        if (wu & (rv | wv) or wv & ru) and ((u[0], u[1]) == (v[0], v[1]) or u not in anc[v]):
            bad.append((u, v))
    return bad


@pytest.mark.parametrize("nz,planes,nsteps", [(128, 16, 3), (32, 16, 4), (48, 16, 3), (40, 16, 3), (72, 24, 3),
                                              (64, 64, 3)])
def test_fused_slab_graph_edges_order_every_conflict(nz, planes, nsteps):
    slabs = _slabs(nz, planes)
    pred = _fused_graph(len(slabs), nsteps)
    acc = {(t, p, i): _fused_accesses(nz, *slabs[i], ("fields", "div", "fused")[p], t) for (t, p, i) in pred}
    assert not _unordered(acc, _ancestors(pred))


def test_fused_model_catches_a_missing_edge():
    """With fused(i) after div(i) alone (the four-pass collision's edge) the
    ring planes of the fused pass would read Q of the next slab before its
    divergence pass writes it."""
    nz, planes = 64, 16
    slabs = _slabs(nz, planes)
    pred = _fused_graph(len(slabs), 2, fused_pred=lambda i: {i})
    acc = {(t, p, i): _fused_accesses(nz, *slabs[i], ("fields", "div", "fused")[p], t) for (t, p, i) in pred}
    assert _unordered(acc, _ancestors(pred))


def _graph(ns, nsteps):
    """Nodes (step, pass, slab) and their predecessor sets, as the library builds them."""
    pred = {}
    near = lambda i: {(i + d) % ns for d in (-1, 0, 1)}
    for t in range(nsteps):
        for i in range(ns):
            pred[(t, 0, i)] = {(t - 1, 3, j) for j in near(i)} if t > 0 else set()
            pred[(t, 1, i)] = {(t, 0, j) for j in near(i)}
            pred[(t, 2, i)] = {(t, 1, j) for j in near(i)}
            pred[(t, 3, i)] = {(t, 2, i)}
    return pred


def _ancestors(pred):
    anc = {}
    for node in sorted(pred):  # (step, pass, slab): predecessors sort first
        a = set()
        for p in pred[node]:
            a |= {p} | anc[p]
        anc[node] = a
    return anc


@pytest.mark.parametrize("mode", ["two_buffers", "in_place"])
@pytest.mark.parametrize("nz,planes,nsteps", [(128, 16, 3), (32, 16, 4), (48, 16, 3), (40, 16, 3), (72, 24, 3)])
def test_slab_graph_edges_order_every_conflict(mode, nz, planes, nsteps):
    slabs = _slabs(nz, planes)
    pred = _graph(len(slabs), nsteps)
    anc = _ancestors(pred)
    acc = {}
    for (t, p, i) in pred:
        zb, ze = slabs[i]
        acc[(t, p, i)] = _accesses(nz, zb, ze, PASSES[p], mode, t)
    nodes = sorted(acc)
    checked = 0
    for u, v in itertools.combinations(nodes, 2):  # u precedes v in sequential order
        ru, wu = acc[u]
        rv, wv = acc[v]
        if not (wu & (rv | wv) or wv & ru):
            continue
        checked += 1
        assert (u[0], u[1]) != (v[0], v[1]), ("two slabs of one pass conflict", u, v)
        assert u in anc[v], ("unordered conflict", u, v)
    assert checked > 0


def test_model_catches_a_missing_edge():
    """Without the cross-step edge to the neighbouring slabs the check fails
    (the next step's pull from slab i-1 would race its collision)."""
    nz, planes = 64, 16
    slabs = _slabs(nz, planes)
    pred = _graph(len(slabs), 2)
    for i in range(len(slabs)):
        pred[(1, 0, i)] = {(0, 3, i)}
    anc = _ancestors(pred)
    acc = {(t, p, i): _accesses(nz, *slabs[i], PASSES[p], "two_buffers", t) for (t, p, i) in pred}
    bad = [(u, v) for u, v in itertools.combinations(sorted(acc), 2)
           if (acc[u][1] & (acc[v][0] | acc[v][1]) or acc[v][1] & acc[u][0]) and u not in anc[v]]
    assert bad


def test_in_place_slot_rules_on_a_3d_lattice():
    """The in-place rules of cg27.h on a periodic 4 x 3 x 5 D3Q27 lattice: in
    each step every slot is read by exactly one cell and written by that same
    cell; and tracing values through an even and an odd step gives the pull
    of the two-buffer scheme (cell x receives, for direction q, the value its
    neighbour x - c_q emitted in the previous step)."""
    nx, ny, nz = 4, 3, 5
    dirs = [(cx, cy, cz) for cz in (-1, 0, 1) for cy in (-1, 0, 1) for cx in (-1, 0, 1)]
    opp = lambda q: 26 - q
    cells = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
    add = lambda a, c, s=1: ((a[0] + s * c[0]) % nx, (a[1] + s * c[1]) % ny, (a[2] + s * c[2]) % nz)
    assert all(dirs[opp(q)] == tuple(-v for v in dirs[q]) for q in range(27))

    def slots(step, cell):
        rd = {q: ((q, cell) if step % 2 == 0 else (opp(q), add(cell, dirs[q], -1))) for q in range(27)}
        wr = {q: ((opp(q), cell) if step % 2 == 0 else (q, add(cell, dirs[q]))) for q in range(27)}
        return rd, wr

    for step in (0, 1):
        readers, writers = {}, {}
        for cell in cells:
            rd, wr = slots(step, cell)
            for s in rd.values():
                readers.setdefault(s, []).append(cell)
            for s in wr.values():
                writers.setdefault(s, []).append(cell)
        assert len(readers) == len(writers) == 27 * len(cells)
        for s, who in readers.items():
            assert len(who) == 1 and writers[s] == who
    # values: before an even step, slot (q, x + c_q) holds what cell x emitted for
    # q (the layout the initialisation writes); run four steps
    mem = {(q, add(cell, dirs[q])): ("init", cell, q) for cell in cells for q in range(27)}
    for step in range(4):
        new = dict(mem)
        for cell in cells:
            rd, wr = slots(step, cell)
            got = {q: mem[rd[q]] for q in range(27)}
            for q in range(27):
                tag, src, qq = got[q]
                assert qq == q and src == add(cell, dirs[q], -1), (step, cell, q, got[q])
                new[wr[q]] = (step, cell, q)
        mem = new
