"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here re-types the oracle's formulas: directions are checked against
hand-worked fixtures, planes and a cone with known answers, and optimality
properties; counts against brute-force path tracing, the local Eq. 1
recursion, conservation and closed forms; the transposed solve against the
adjoint identity, finite differences and brute-force path sums.
"""
import math

import numpy as np
import pytest

import demgen
import oracle
from tests import brute
from tests.golden_io import grid, named, sections

RULES = ("steepest", "lowest")


# --------------------------------------------------------------- directions
def test_golden_3x3_cases():
    cases = sections("flowdir_3x3_cases.txt")
    zs = [rows for h, rows in cases if h == "case"]
    cs = [rows for h, rows in cases if h == "centre"]
    assert len(zs) == len(cs) == 7
    for z_rows, c_rows in zip(zs, cs):
        z = grid(z_rows, np.float32)
        want = [int(x) for x in c_rows[0]]
        for rule, w in zip(RULES, want):
            d = oracle.flowdir(z, rule)
            assert d[1, 1] == w, (rule, z, d)
            border = np.ones_like(d, dtype=bool)
            border[1, 1] = False
            assert (d[border] == oracle.OUTLET).all()


def test_golden_5x5_directions_and_counts():
    g = named("grid_5x5.txt")
    z = grid(g["z"], np.float32)
    for rule in RULES:
        d = oracle.flowdir(z, rule)
        np.testing.assert_array_equal(d, grid(g[f"dir {rule}"], np.uint8))
        np.testing.assert_array_equal(oracle.accumulate(d), grid(g[f"count {rule}"], np.uint32))
    d = oracle.flowdir(z, "steepest")
    w = np.repeat(np.arange(1, 6, dtype=np.float64)[:, None], 5, axis=1)
    np.testing.assert_array_equal(oracle.accumulate_weighted(d, w), grid(g["weighted steepest"], np.float64))
    np.testing.assert_array_equal(oracle.transposed(d, np.ones((5, 5))), grid(g["pathlen steepest"], np.float64))
    e = np.zeros((5, 5))
    e[3, 2] = 1.0
    np.testing.assert_array_equal(oracle.transposed(d, e), grid(g["upslope32 steepest"], np.float64))


def test_golden_4x5_counts():
    g = named("counts_4x5_dirs.txt")
    d = grid(g["dir"], np.uint8)
    np.testing.assert_array_equal(oracle.accumulate(d), grid(g["count"], np.uint32))


@pytest.mark.parametrize("code", range(8))
@pytest.mark.parametrize("rule", RULES)
def test_planes_pin_each_code(code, rule):
    """A plane descending along direction k drains every interior cell to k
    (steepest).  Under the lowest rule a plane descending along a cardinal
    direction has three equally low neighbours (the cardinal and its two
    diagonals), so the first of them in N,NE,...,NW order is taken."""
    di = (-1, -1, 0, 1, 1, 1, 0, -1)[code]
    dj = (0, 1, 1, 1, 0, -1, -1, -1)[code]
    H, W = 9, 11
    i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    z = (-(di * i + dj * j) + 3 * (H + W)).astype(np.float32)
    d = oracle.flowdir(z, rule)
    want = code if (rule == "steepest" or code % 2) else {0: 0, 2: 1, 4: 3, 6: 5}[code]
    assert (d[1:-1, 1:-1] == want).all()
    assert (d[0] == 8).all() and (d[-1] == 8).all() and (d[:, 0] == 8).all() and (d[:, -1] == 8).all()


def test_cone_rays():
    """On a cone the cells on the eight rays from the apex drain along the ray
    (steepest rule; the lowest rule follows the four diagonal rays only, since
    off a cardinal ray the diagonal neighbour is farther from the apex)."""
    n = 21
    c = n // 2
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    z = (100.0 - np.sqrt((i - c) ** 2 + (j - c) ** 2)).astype(np.float32)
    for rule in RULES:
        d = oracle.flowdir(z, rule)
        for code, (di, dj) in enumerate(zip((-1, -1, 0, 1, 1, 1, 0, -1), (0, 1, 1, 1, 0, -1, -1, -1))):
            if rule == "lowest" and code % 2 == 0:
                continue
            for r in range(1, c):
                assert d[c + r * di, c + r * dj] == code, (rule, code, r)


@pytest.mark.parametrize("rule", RULES)
def test_direction_optimality(rule):
    """Every interior non-SINK cell drains to a strictly lower neighbour, and no
    neighbour beats the chosen one (ties only with a later neighbour)."""
    z = demgen.fractal(96, 80, seed=7, cache=False)
    d = oracle.flowdir(z, rule)
    R = np.float32(np.frombuffer(np.uint32(0x3F3504F3).tobytes(), dtype=np.float32)[0])
    assert abs(float(R) - 1 / math.sqrt(2)) < 1e-7
    DI = (-1, -1, 0, 1, 1, 1, 0, -1)
    DJ = (0, 1, 1, 1, 0, -1, -1, -1)
    H, W = z.shape
    for a in range(1, H - 1):
        for b in range(1, W - 1):
            k = int(d[a, b])
            assert k < 8  # filled DEM: no sinks
            zc = z[a, b]
            assert z[a + DI[k], b + DJ[k]] < zc
            if rule == "steepest":
                s = [np.float32(zc - z[a + DI[m], b + DJ[m]]) * (R if m % 2 else np.float32(1)) for m in range(8)]
                best = s[k]
                for m in range(8):
                    assert s[m] <= best
                    if s[m] == best:
                        assert m >= k
            else:
                for m in range(8):
                    zn = z[a + DI[m], b + DJ[m]]
                    assert zn >= z[a + DI[k], b + DJ[k]]
                    if zn == z[a + DI[k], b + DJ[k]]:
                        assert m >= k


def test_nonfinite_flagged():
    z = demgen.fractal(16, 16, seed=3, cache=False)
    z[5, 5] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.flowdir(z)
    assert e.value.code == oracle.ERR_NONFINITE
    d = oracle.flowdir(z, allow_nonfinite=True)
    assert d[5, 5] == oracle.SINK


# ------------------------------------------------------------------- counts
@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("rule", RULES)
def test_counts_match_bruteforce_fractal(seed, rule):
    H, W = 48 + 7 * seed, 64 - 5 * seed
    z = demgen.fractal(H, W, seed=seed, cache=False)
    d = oracle.flowdir(z, rule)
    np.testing.assert_array_equal(oracle.accumulate(d), brute.counts(d).astype(np.uint32))


@pytest.mark.parametrize("seed", range(6))
def test_counts_match_bruteforce_random_dirs(seed):
    """Arbitrary direction fields (codes 0..9, off-grid targets end paths)."""
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    # bias towards acyclic fields: mostly S/SE/SW/E with some terminals
    d = rng.choice(np.array([2, 3, 4, 5, 8, 9], dtype=np.uint8), size=(H, W), p=[.2, .2, .3, .2, .05, .05])
    b = brute.counts(d)
    if b is None:
        with pytest.raises(oracle.OracleError):
            oracle.accumulate(d)
    else:
        np.testing.assert_array_equal(oracle.accumulate(d), b.astype(np.uint32))


@pytest.mark.parametrize("seed", range(8))
def test_cycles_agree_with_bruteforce(seed):
    d = demgen.random_dirs(12, 13, seed=100 + seed)
    b = brute.counts(d)
    if b is None:
        with pytest.raises(oracle.OracleError) as e:
            oracle.accumulate(d)
        assert e.value.code == oracle.ERR_CYCLE
    else:
        np.testing.assert_array_equal(oracle.accumulate(d), b.astype(np.uint32))


def test_two_cycle_detected():
    d = np.full((3, 4), 8, dtype=np.uint8)
    d[1, 1], d[1, 2] = 2, 6  # E then W: a 2-cycle
    with pytest.raises(oracle.OracleError) as e:
        oracle.accumulate(d)
    assert e.value.code == oracle.ERR_CYCLE


def test_invalid_code_rejected():
    d = np.full((3, 3), 8, dtype=np.uint8)
    d[1, 1] = 12
    with pytest.raises(oracle.OracleError) as e:
        oracle.accumulate(d)
    assert e.value.code == oracle.ERR_ARG


@pytest.mark.parametrize("rule", RULES)
def test_recursion_and_conservation(rule):
    """Eq. 1 holds at every cell; the terminals collect every cell once."""
    z = demgen.fractal(512, 384, seed=11)
    d = oracle.flowdir(z, rule)
    A = oracle.accumulate(d)
    assert brute.recursion_residual(d, A) == 0
    term = brute.terminal_mask(d)
    assert int(A[term].astype(np.int64).sum()) == z.size
    assert (A >= 1).all()


def test_tilted_plane_closed_form():
    """Noise-free plane falling due S.  Steepest: every interior cell drains S,
    so A(i, j) = i in the interior and the bottom edge collects H - 1.  Lowest:
    S, SE and SW tie, SE comes first, so flow runs down the diagonals and
    A(i, j) = min(i, j) in the interior; an edge cell below/right of the
    interior collects its diagonal chain plus itself."""
    H, W = 37, 29
    z = demgen.plane_exact(H, W, sy=1.0, sx=0.0)
    d = oracle.flowdir(z, "steepest")
    assert (d[1:-1, 1:-1] == 4).all()
    A = oracle.accumulate(d).astype(np.int64)
    want = np.ones((H, W), dtype=np.int64)
    want[1:-1, 1:-1] = np.arange(1, H - 1)[:, None]
    want[-1, 1:-1] = H - 1
    np.testing.assert_array_equal(A, want)

    d = oracle.flowdir(z, "lowest")
    assert (d[1:-1, 1:-1] == 3).all()
    A = oracle.accumulate(d).astype(np.int64)
    want = np.ones((H, W), dtype=np.int64)
    i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    want[1:-1, 1:-1] = np.minimum(i, j)[1:-1, 1:-1]
    for jj in range(2, W):  # bottom edge: fed by (H-2, jj-1)
        want[H - 1, jj] = 1 + min(H - 2, jj - 1)
    for ii in range(2, H):  # right edge: fed by (ii-1, W-2)
        want[ii, W - 1] = 1 + min(ii - 1, W - 2)
    np.testing.assert_array_equal(A, want)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (6, 1), (5, 8), (64, 33)])
def test_serpentine_closed_form(shape):
    H, W = shape
    d = demgen.serpentine_dirs(H, W)
    A = oracle.accumulate(d).astype(np.int64)
    # walk the boustrophedon order: the k-th cell on the path has A = k + 1
    k = 0
    for i in range(H):
        cols = range(W) if i % 2 == 0 else range(W - 1, -1, -1)
        for j in cols:
            assert A[i, j] == k + 1
            k += 1


def test_degenerate_shapes_are_all_outlets():
    for H, W in [(1, 1), (1, 5), (2, 2), (2, 9), (7, 2)]:
        z = np.random.default_rng(0).random((H, W)).astype(np.float32)
        d = oracle.flowdir(z)
        assert (d == oracle.OUTLET).all()
        assert (oracle.accumulate(d) == 1).all()


# ----------------------------------------------------------------- weighted
def test_weighted_matches_bruteforce_and_linearity():
    z = demgen.fractal(40, 52, seed=5, cache=False)
    d = oracle.flowdir(z)
    w1 = demgen.lognormal_weights(40, 52, seed=1).astype(np.float64)
    w2 = demgen.lognormal_weights(40, 52, seed=2).astype(np.float64)
    A1 = oracle.accumulate_weighted(d, w1)
    np.testing.assert_allclose(A1, brute.counts(d, w1), rtol=1e-12)
    A12 = oracle.accumulate_weighted(d, w1 + w2)
    np.testing.assert_allclose(A12, A1 + oracle.accumulate_weighted(d, w2), rtol=1e-12)
    assert brute.recursion_residual(d, A1, w1) < 1e-9
    np.testing.assert_array_equal(oracle.accumulate_weighted(d, np.ones_like(w1)), oracle.accumulate(d))


# --------------------------------------------------------------- transposed
def test_transposed_adjoint_identity_and_bruteforce():
    z = demgen.fractal(60, 44, seed=9, cache=False)
    d = oracle.flowdir(z)
    w = demgen.lognormal_weights(60, 44, seed=3).astype(np.float64)
    c = demgen.normal_cotangent(60, 44, seed=4).astype(np.float64)
    G = oracle.transposed(d, c)
    A = oracle.accumulate_weighted(d, w)
    lhs, rhs = float((c * A).sum()), float((G * w).sum())
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + abs(rhs))
    np.testing.assert_allclose(G, brute.path_sums(d, c), rtol=1e-12, atol=1e-12)
    # c = 1: path lengths; c = e_p: indicator of p's up-slope set
    plen = np.array([len(p) for p in brute.paths(d)]).reshape(d.shape)
    np.testing.assert_array_equal(oracle.transposed(d, np.ones_like(c)), plen)
    p = (30, 20)
    e = np.zeros_like(c)
    e[p] = 1.0
    up = np.array([p[0] * d.shape[1] + p[1] in q for q in brute.paths(d)]).reshape(d.shape)
    np.testing.assert_array_equal(oracle.transposed(d, e), up.astype(np.float64))


def test_transposed_central_differences():
    """L(w) = sum c*A(w) is linear in w, so a central difference with h = 1
    gives dL/dw exactly up to rounding."""
    H, W = 48, 40
    z = demgen.fractal(H, W, seed=12, cache=False)
    d = oracle.flowdir(z)
    w = demgen.lognormal_weights(H, W, seed=5).astype(np.float64)
    c = demgen.normal_cotangent(H, W, seed=6).astype(np.float64)
    G = oracle.transposed(d, c)
    rng = np.random.default_rng(7)
    for q in rng.choice(H * W, size=64, replace=False):
        e = np.zeros(H * W)
        e[q] = 1.0
        e = e.reshape(H, W)
        Lp = float((c * oracle.accumulate_weighted(d, w + e)).sum())
        Lm = float((c * oracle.accumulate_weighted(d, w - e)).sum())
        fd = (Lp - Lm) / 2.0
        assert abs(fd - G.ravel()[q]) <= 1e-9 * max(1.0, abs(fd))


# ------------------------------------------------------------ epsilon fill
def _fill_fixed_point_residual(z, F, eps):
    """Cells where F breaks the fill's defining equations (an independent
    restatement of them in numpy): F = z on the edge; inside, with m the
    lowest of the 8 neighbouring F, F = z if z > m else max(m + eps, next fp32
    above m)."""
    z = z.astype(np.float32)
    H, W = z.shape
    bad = np.zeros((H, W), dtype=bool)
    edge = np.zeros((H, W), dtype=bool)
    edge[0, :] = edge[-1, :] = edge[:, 0] = edge[:, -1] = True
    bad |= edge & (F != z)
    if H >= 3 and W >= 3:
        Fp = np.pad(F, 1, constant_values=np.inf)
        m = np.full((H, W), np.inf, dtype=np.float32)
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                if di or dj:
                    m = np.minimum(m, Fp[1 + di:1 + di + H, 1 + dj:1 + dj + W])
        up = np.maximum((m + np.float32(eps)).astype(np.float32), np.nextafter(m, np.float32(np.inf)))
        want = np.where(z > m, z, up)
        bad |= ~edge & (F != want)
    return bad


def _fill_by_iteration(z, eps):
    """Brute force for tiny grids: start from +inf inside and apply the
    defining equations to every interior cell until nothing changes (a
    different algorithm from the oracle's priority flood)."""
    z = z.astype(np.float32)
    H, W = z.shape
    F = np.full((H, W), np.inf, dtype=np.float32)
    F[0, :], F[-1, :], F[:, 0], F[:, -1] = z[0, :], z[-1, :], z[:, 0], z[:, -1]
    for _ in range(10 * H * W):
        changed = False
        for i in range(1, H - 1):
            for j in range(1, W - 1):
                m = min(F[i + di, j + dj] for di in (-1, 0, 1) for dj in (-1, 0, 1) if di or dj)
                m = np.float32(m)
                v = z[i, j] if z[i, j] > m else max(np.float32(m + np.float32(eps)), np.nextafter(m, np.float32(np.inf)))
                if v != F[i, j]:
                    F[i, j] = v
                    changed = True
        if not changed:
            return F
    raise AssertionError("iteration did not settle")


def test_fill_golden_cases():
    g = named("fill_cases.txt")
    for name in ("bowl", "plateau", "spill", "keep", "step"):
        rows = g[name]
        eps = float(rows[0][0])
        z = grid(rows[1:], np.float32)
        F = oracle.fill_eps(z, eps)
        np.testing.assert_array_equal(F, grid(g[name + "_F"], np.float32), err_msg=name)


def test_fill_matches_iteration_on_tiny_grids():
    rng = np.random.default_rng(1605)
    for k in range(30):
        H, W = int(rng.integers(1, 8)), int(rng.integers(1, 9))
        z = rng.integers(0, 5, size=(H, W)).astype(np.float32)  # many ties and flats
        eps = [0.25, 0.001, 0.0][k % 3]
        np.testing.assert_array_equal(oracle.fill_eps(z, eps), _fill_by_iteration(z, eps), err_msg=f"case {k}")


def test_fill_defining_equations_and_properties():
    cases = [demgen.fractal_raw(257, 300, 5), demgen.fractal_raw(129, 65, 6),
             np.random.default_rng(3).random((97, 131)).astype(np.float32) * 10]
    for z in cases:
        F = oracle.fill_eps(z, 1e-3)
        assert not _fill_fixed_point_residual(z, F, 1e-3).any()
        assert (F >= z).all()
        # every interior cell drains: it has a strictly lower neighbour, so the
        # steepest and lowest rules give no SINK
        for rule in RULES:
            assert not (oracle.flowdir(F, rule) == 9).any()
        np.testing.assert_array_equal(oracle.fill_eps(F, 1e-3), F)  # idempotent
    z = demgen.fractal(200, 180, seed=8, cache=False)  # already drains everywhere: unchanged
    np.testing.assert_array_equal(oracle.fill_eps(z, 1e-3), z)


def test_fill_rejects_nonfinite():
    z = np.zeros((5, 5), dtype=np.float32)
    z[2, 2] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.fill_eps(z)


# ------------------------------------------------------------ NODATA masks
def test_nodata_golden_and_properties():
    g = named("nodata_6x6.txt")
    z = grid(g["z"], np.float32)
    for rule in ("steepest_nodata", "lowest_nodata"):
        np.testing.assert_array_equal(oracle.flowdir(z, rule), grid(g[rule], np.uint8), err_msg=rule)
    # away from holes the mask changes nothing; every hole and every cell next
    # to one is OUTLET; no error for the non-finite cells
    rng = np.random.default_rng(20)
    z = demgen.fractal(120, 97, seed=21, cache=False)
    holes = rng.random(z.shape) < 0.03
    z[holes] = np.nan
    z[40:60, 30:50] = np.nan  # a lake
    near = holes.copy()
    near[40:60, 30:50] = True
    pad = np.pad(near, 1)
    touch = np.zeros_like(near)
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            touch |= pad[1 + di:1 + di + z.shape[0], 1 + dj:1 + dj + z.shape[1]]
    for rule in RULES:
        d = oracle.flowdir(z, rule + "_nodata")
        assert (d[touch] == 8).all()
        plain = oracle.flowdir(z, rule, allow_nonfinite=True)
        np.testing.assert_array_equal(d[~touch], plain[~touch])
        A = oracle.accumulate(d)  # a valid field: no cycle, conservation holds
        assert int(A.astype(np.int64)[d >= 8].sum()) + int(
            A.astype(np.int64)[(d < 8) & _off_grid_targets(d)].sum()) == z.size


def _off_grid_targets(d):
    H, W = d.shape
    i, j = np.indices(d.shape)
    DI = np.array([-1, -1, 0, 1, 1, 1, 0, -1])
    DJ = np.array([0, 1, 1, 1, 0, -1, -1, -1])
    k = np.minimum(d, 7)
    ti, tj = i + DI[k], j + DJ[k]
    return (ti < 0) | (tj < 0) | (ti >= H) | (tj >= W)
