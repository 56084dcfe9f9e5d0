"""Plant plausible mistakes in a COPY of the oracle source and check that the
pins catch each one (the mistakes live only in a temporary build on the CPU)."""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

MUTATIONS = {
    # the diagonal slope loses its 1/sqrt(2) distance factor
    "no_diagonal_distance": ("float slope = (k & 1) ? drop * R : drop;", "float slope = drop;"),
    # ties go to the LAST direction instead of the first
    "tie_to_last": ("if (slope > best) {", "if (slope >= best) {"),
    # NE and NW swapped in the neighbour table
    "ne_nw_swapped": ("static const int ODJ[8] = {0, 1, 1, 1, 0, -1, -1, -1};",
                      "static const int ODJ[8] = {0, -1, 1, 1, 0, -1, -1, 1};"),
    # the cell's own unit weight dropped from Eq. 1
    "dropped_unit_term": ("uint64_t a = 1;", "uint64_t a = 0;"),
    # the weighted form uses 1 instead of w(c)
    "weight_ignored": ("double a = w ? w[c] : 1.0;", "double a = 1.0;"),
    # the transposed solve drops the cell's own coefficient
    "adjoint_dropped_term": ("G[q] = cvec[q] + (s >= 0 ? G[s] : 0.0);", "G[q] = (s >= 0 ? G[s] : 0.0);"),
    # the transposed solve runs in the forward order (wrong dependency order)
    "adjoint_wrong_order": ("for (int64_t t = N - 1; t >= 0; t--) {", "for (int64_t t = 0; t < N; t++) {"),
    # the lowest rule keeps the HIGHEST lower neighbour
    "lowest_inverted": ("if (zn < best) {", "if (zn < zc && (best == zc || zn > best)) {"),
    # the fill keeps a cell level with its lowest neighbour (flats not resolved)
    "fill_keeps_flats": ("F[c] = z[c] > p.f ? z[c] : fill_up(p.f, eps);",
                         "F[c] = z[c] >= p.f ? z[c] : fill_up(p.f, eps);"),
    # the raise loses its one-step minimum (x + eps can round back to x)
    "fill_no_min_step": ("return a > b ? a : b;", "return a;"),
    # the NODATA mask forgets the study area's edge (cells next to a hole)
    "nodata_edge_missed": ("for (int k = 0; k < 8; k++) hole |= !isfinite(z[(i + ODI[k]) * W + (j + ODJ[k])]);",
                           ""),
    # the flood pops the HIGHEST cell first
    "fill_heap_inverted": ("return a.f < b.f || (a.f == b.f && a.c < b.c);",
                           "return a.f > b.f || (a.f == b.f && a.c < b.c);"),
}

PINS = [
    pins.test_golden_3x3_cases,
    pins.test_golden_5x5_directions_and_counts,
    pins.test_golden_4x5_counts,
    lambda: [pins.test_planes_pin_each_code(k, r) for k in range(8) for r in pins.RULES],
    pins.test_cone_rays,
    pins.test_weighted_matches_bruteforce_and_linearity,
    pins.test_transposed_adjoint_identity_and_bruteforce,
    pins.test_fill_golden_cases,
    pins.test_nodata_golden_and_properties,
    pins.test_fill_matches_iteration_on_tiny_grids,
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) >= 1, name
    path = os.path.join(tmp_path, "mutant.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(tmp_path, "libmutant.so")
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-shared", "-fPIC", "-o", so, path, "-lm"])
    caught = []
    with oracle.use_library(so):
        for pin in PINS:
            try:
                pin()
            except Exception:  # any failing pin counts, whatever it raises
                caught.append(pin)
    assert caught, f"mutation {name} was not caught by any pin"
