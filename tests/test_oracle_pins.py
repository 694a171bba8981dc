"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

None of these values comes from the oracle itself or from the CUDA library:
closed forms of BC on textbook graphs (Eq. 1 evaluated by hand), exact
brute-force enumeration of shortest paths (Eq. 1 with rationals), path
counts that equal binomial coefficients, the path-length identity of Brandes'
dependencies, and invariances (relabelling, s-t symmetry, source
multiplicity).  Each pin is chosen so that a plausible slip in the oracle
(a dropped "1 +" in Eq. 2, a flipped ratio, a missing v != s test, an
off-by-one level, a lost carry in sigma) fails at least one of them; the
mutation test at the end checks exactly that.
"""
import math
import os
import random
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.brute import brute_bc
from paper_2008_05718_gb300 import graphgen as gg

REL = 1e-12


def all_bc(g):
    b, _ = oracle.bc_graph(g, np.arange(g.n))
    return b


# ---- closed forms (Eq. 1 by hand, ordered pairs) -----------------------------

@pytest.mark.parametrize("n", [2, 3, 4, 5, 9, 16])
def test_path(n):
    b = all_bc(gg.path(n))
    assert np.array_equal(b, [2 * i * (n - 1 - i) for i in range(n)])


@pytest.mark.parametrize("n", [2, 3, 6, 11])
def test_star(n):
    b = all_bc(gg.star(n))
    assert b[0] == (n - 1) * (n - 2) and np.all(b[1:] == 0)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 10, 13])
def test_cycle(n):
    b = all_bc(gg.cycle(n))
    want = (n - 1) * (n - 3) / 4 if n % 2 else (n - 2) ** 2 / 4
    assert np.allclose(b, want, rtol=REL, atol=0)


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_complete(n):
    assert np.all(all_bc(gg.complete(n)) == 0)


@pytest.mark.parametrize("a,b", [(1, 4), (2, 3), (3, 4), (5, 2)])
def test_complete_bipartite(a, b):
    # side-A vertex: b(b-1) ordered B-B pairs at distance 2, a middle choices each
    bc = all_bc(gg.complete_bipartite(a, b))
    assert np.allclose(bc[:a], b * (b - 1) / a, rtol=REL, atol=0)
    assert np.allclose(bc[a:], a * (a - 1) / b, rtol=REL, atol=0)


def diamond_closed_form(k):
    want = np.zeros(3 * k + 1)
    for i in range(k + 1):
        want[3 * i] = 1 if i in (0, k) else 18 * i * (k - i) + 2
    for i in range(1, k + 1):
        want[3 * i - 2] = want[3 * i - 1] = (3 * i - 2) * (3 * k - 3 * i + 1)
    if k == 0:
        want[0] = 0
    return want


@pytest.mark.parametrize("k", [1, 2, 3, 8, 63, 64, 65, 100])
def test_diamond_chain_bc(k):
    # every sigma in a diamond chain is a power of two, so the arithmetic is
    # exact even when sigma passes 2^64: BC must equal the closed form exactly
    g = gg.diamond_chain(k)
    assert np.array_equal(all_bc(g), diamond_closed_form(k))


@pytest.mark.parametrize("k", [62, 63, 64, 65, 100, 130])
def test_diamond_chain_sigma_overflow(k):
    g = gg.diamond_chain(k)
    _, st = oracle.bc_graph(g, [0], dump=[0])
    s = st[0]
    for i in range(k + 1):
        true = 1 << i  # sigma(c_0 -> c_i)
        assert s.dist[3 * i] == 2 * i
        assert int(s.sigma[3 * i]) == true % (1 << 64)
        assert s.ovf[3 * i] == (true >= 1 << 64)
    for i in range(1, k + 1):
        true = 1 << (i - 1)  # sigma(c_0 -> a_i) = sigma(c_0 -> c_{i-1})
        assert int(s.sigma[3 * i - 2]) == true % (1 << 64) and s.ovf[3 * i - 2] == (true >= 1 << 64)


@pytest.mark.parametrize("rows,cols", [(8, 8), (40, 40), (3, 70)])
def test_full_grid_sigma_binomial(rows, cols):
    # shortest corner paths in a full grid are lattice paths: sigma = C(i+j, i)
    g = gg.full_grid(rows, cols)
    _, st = oracle.bc_graph(g, [0], dump=[0])
    s = st[0]
    for i in range(rows):
        for j in range(cols):
            v = i * cols + j
            c = math.comb(i + j, i)
            assert s.dist[v] == i + j
            assert int(s.sigma[v]) == c % (1 << 64)
            assert s.ovf[v] == (c >= 1 << 64)


def test_full_grid_delta_path_identity_with_overflow():
    # 40x40 grid from a corner: sigma reaches C(78, 39) > 2^64 (wide sigma)
    g = gg.full_grid(40, 40)
    _, st = oracle.bc_graph(g, [0], dump=[0])
    s = st[0]
    want = sum(d - 1 for d in s.dist if d >= 1)
    assert s.ovf.any()
    assert math.isclose(s.delta[s.dist != 0].sum(), want, rel_tol=REL)


# ---- brute force on random small graphs (Eq. 1, exact rationals) ------------

def random_graphs(count, seed):
    r = random.Random(seed)
    for _ in range(count):
        n = r.randint(1, 10)
        p = r.choice([0.15, 0.3, 0.45, 0.6])
        # cap density for n = 10 to keep path enumeration quick
        if n >= 9:
            p = min(p, 0.35)
        edges = [(u, v) for u in range(n) for v in range(u + 1, n) if r.random() < p]
        yield n, edges


def test_brute_force_random_graphs():
    checked = disconnected = 0
    for n, edges in random_graphs(200, seed=20080571):
        g = gg.from_edges(n, edges if edges else np.zeros((0, 2), np.int32))
        srcs = list(range(n))
        b, st = oracle.bc_graph(g, srcs, dump=srcs)
        bb, dist, sig = brute_bc(n, edges)
        for v in range(n):
            assert math.isclose(b[v], float(bb[v]), rel_tol=REL, abs_tol=1e-15), (n, edges, v)
        for s in srcs:
            assert list(st[s].dist) == dist[s]
            assert [int(x) for x in st[s].sigma] == sig[s]
            assert not st[s].ovf.any()
        comps = len({min(t for t in range(n) if dist[s][t] >= 0) for s in srcs})
        disconnected += comps > 1
        checked += 1
    assert checked == 200 and disconnected > 20


def test_brute_force_source_subset_and_multiplicity():
    n, edges = 9, [(0, 1), (1, 2), (2, 3), (1, 4), (4, 3), (3, 5), (5, 6), (6, 7), (5, 7), (7, 8)]
    g = gg.from_edges(n, edges)
    S = [3, 1, 3, 8]
    b, _ = oracle.bc_graph(g, S)
    bb, _, _ = brute_bc(n, edges, S)
    assert np.allclose(b, [float(x) for x in bb], rtol=REL, atol=1e-15)


# ---- identities and invariances ---------------------------------------------

def check_path_length_identity(g, sources):
    # sum over v != s of delta_s(v) = sum over reachable t != s of (d(s,t) - 1):
    # every shortest s-t path has d(s,t) - 1 interior vertices, each counted
    # 1/sigma_st (the recurrence's value at v = s itself is not a dependency)
    _, st = oracle.bc_graph(g, sources, dump=range(len(sources)))
    for i in range(len(sources)):
        d = st[i].dist
        want = float(np.sum(d[d >= 1] - 1))
        got = float(np.sum(st[i].delta[d != 0]))
        assert math.isclose(got, want, rel_tol=REL, abs_tol=1e-9), (i, got, want)


def test_path_length_identity_er():
    g = gg.er(300, Fraction(6, 299), seed=7)
    check_path_length_identity(g, [0, 5, 17, 299])


def test_path_length_identity_rmat():
    g = gg.rmat(10, 16, seed=11)
    check_path_length_identity(g, list(gg.sample_sources(g.n, 8, seed=11)))


def test_path_length_identity_grid_with_overflow():
    g = gg.grid(48, "0.05", seed=13)
    check_path_length_identity(g, list(gg.sample_sources(g.n, 3, seed=13)))


def test_bc_sum_identity_er4096_all_sources():
    # the config-1 workload in full: sum_v BC(v) = sum_s sum_t (d(s,t) - 1)
    g, S = gg.workload("er4096")
    b, st = oracle.bc_graph(g, S[:512], dump=range(512))
    want = sum(float(np.sum(st[i].dist[st[i].dist >= 1] - 1)) for i in range(512))
    assert math.isclose(b.sum(), want, rel_tol=REL)


def test_relabel_invariance():
    g = gg.rmat(9, 8, seed=21)
    perm = gg.permutation(g.n, seed=22)
    h = gg.relabel(g, perm)
    S = np.arange(0, g.n, 7, dtype=np.int32)
    bg, _ = oracle.bc_graph(g, S)
    bh, _ = oracle.bc_graph(h, perm[S])
    assert np.allclose(bh[perm], bg, rtol=REL, atol=1e-12)


def test_st_symmetry_all_sources():
    g = gg.er(120, Fraction(3, 119), seed=5)
    S = list(range(g.n))
    _, st = oracle.bc_graph(g, S, dump=S)
    D = np.stack([st[s].dist for s in S])
    G = np.stack([st[s].sigma for s in S])
    assert np.array_equal(D, D.T) and np.array_equal(G, G.T)


def test_unreachable_and_isolated():
    g = gg.from_edges(7, [(0, 1), (1, 2), (4, 5)])  # 3 and 6 isolated
    b, st = oracle.bc_graph(g, [0, 3, 4], dump=[0, 1, 2])
    assert list(st[0].dist) == [0, 1, 2, -1, -1, -1, -1]
    assert list(st[1].dist) == [-1, -1, -1, 0, -1, -1, -1]
    assert list(st[1].sigma) == [0, 0, 0, 1, 0, 0, 0]
    assert np.array_equal(b, [0, 1, 0, 0, 0, 0, 0])


def test_leaves_have_zero_bc():
    g = gg.rmat(8, 4, seed=3)
    b = all_bc(g)
    leaves = np.flatnonzero(g.degrees() == 1)
    assert len(leaves) > 0 and np.all(b[leaves] == 0)


def test_duplicate_sources_counted_twice():
    g = gg.er(200, Fraction(5, 199), seed=9)
    S = [3, 50, 199]
    b1, _ = oracle.bc_graph(g, S)
    b2, _ = oracle.bc_graph(g, S + S)
    assert np.allclose(b2, 2 * b1, rtol=REL, atol=0)


def test_invalid_source_rejected():
    g = gg.path(4)
    with pytest.raises(ValueError):
        oracle.bc_graph(g, [4])


# ---- the rounding helper against CPython's correctly rounded int -> float ---

def test_big_to_scaled_correct_rounding():
    r = random.Random(1)
    cases = [0, 1, 2, 3, (1 << 53) - 1, 1 << 53, (1 << 53) + 1, (1 << 54) + 2, (1 << 54) + 6,
             (1 << 64) - 1, 1 << 64, (1 << 64) + 1, (1 << 1023), (1 << 1024) - 1]
    for bits in [54, 60, 64, 65, 100, 127, 128, 129, 500, 1000, 1023]:
        for _ in range(40):
            cases.append(r.getrandbits(bits) | (1 << (bits - 1)))
        # exact ties, with and without sticky bits below the tie bit
        base = (r.getrandbits(52) | (1 << 52)) << (bits - 53)
        cases += [base + (1 << (bits - 54)), base + (1 << (bits - 54)) + 1, base + (1 << (bits - 53)) + (1 << (bits - 54))]
    for x in cases:
        m, e = oracle.big_to_scaled(x)
        if x < (1 << 1024) - (1 << 970):
            assert math.ldexp(m, e) == float(x), x
        if x:
            assert 1.0 <= m < 2.0


def test_big_to_scaled_beyond_double_range():
    # 3 * 2^1500 + tie/sticky patterns: compare with the exact rational rounding
    for x in [3 << 1500, (3 << 1500) + 1, ((1 << 53) - 1) << 2000, (((1 << 53) - 1) << 2000) + (1 << 1999)]:
        m, e = oracle.big_to_scaled(x)
        b = x.bit_length()
        exact = Fraction(x, 1 << (b - 1))  # in [1, 2)
        assert e == b - 1 or (e == b and m == 1.0)
        got = Fraction(m) * (2 if e == b else 1)
        assert abs(got - exact) <= Fraction(1, 1 << 53)


# ---- mutation check: the pins above catch plausible oracle slips ------------

MUTANTS = {
    "drop_one_plus": ("* (1.0 + delta[u])", "* (delta[u])"),
    "flip_ratio": ("ldexp(mv / mu, (int)d)", "ldexp(mu / mv, (int)-d)"),
    "count_source": ("if (v != s) bc[v] += delta[v];", "bc[v] += delta[v];"),
    "skip_deepest_level": ("int32_t cur = nlev - 1;", "int32_t cur = nlev - 2;"),
    "lose_carry": ("carry = c1 | c2;", "carry = 0;"),
    "ties_away": ("(rem == 0x400ULL && (sticky || (keep & 1)))", "(rem == 0x400ULL)"),
    "pred_any_level": ("if (dist[w] == dist[v] + 1) {", "if (dist[w] >= dist[v]) {"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    """Compile a copy of the oracle with one planted mistake (on the CPU) and
    check that at least one pin-style check fails on it."""
    import ctypes
    src = open(os.path.join(os.path.dirname(oracle.__file__), "brandes.c")).read()
    a, b = MUTANTS[name]
    assert a in src, name
    p = tmp_path / "m.c"
    p.write_text(src.replace(a, b))
    so = tmp_path / "m.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-o", str(so), str(p), "-lm"])
    lib = ctypes.CDLL(str(so))
    lib.oracle_bc.argtypes = oracle._load().oracle_bc.argtypes
    lib.oracle_big_to_scaled.argtypes = oracle._load().oracle_big_to_scaled.argtypes
    lib.oracle_big_to_scaled.restype = None
    saved = oracle._lib
    try:
        oracle._lib = lib
        failed = False
        for check in (lambda: test_path(9), lambda: test_diamond_chain_bc(65),
                      lambda: test_diamond_chain_sigma_overflow(65), test_brute_force_random_graphs,
                      test_path_length_identity_er, test_full_grid_delta_path_identity_with_overflow,
                      test_big_to_scaled_correct_rounding):
            try:
                check()
            except AssertionError:
                failed = True
                break
        assert failed, f"mutant {name} survived every pin"
    finally:
        oracle._lib = saved
