"""The roofline figures of the benchmark line rest on two per-element counts:
the algorithmic DRAM bytes of one fused LSERK stage (averaged over the five
stages of a step) and the algorithmic flops of the FP32 form. These tests count
them stage by stage and term by term from the definition and compare with the
helpers the benchmark uses."""
import pytest

import bench


def _stage_bytes(N, Npad):
    """Bytes of each of the five LSERK4 stages: u read, res read (not in the
    first stage, whose coefficient a_1 is zero), res and u_out written, FP32,
    six fields; plus per element 64 B of geometry, 4 x 16 B of face geometry
    and 4 x 8 B of face connectivity."""
    field = 6 * Npad * 4
    per_stage = []
    for s in range(5):
        vectors = 1 + (0 if s == 0 else 1) + 2
        per_stage.append(vectors * field + 64 + 4 * 16 + 4 * 8)
    return per_stage


@pytest.mark.parametrize("N, Npad", [(1, 4), (3, 20), (4, 36), (5, 56), (7, 120)])
def test_bytes_per_element_is_the_five_stage_mean(N, Npad):
    stages = _stage_bytes(N, Npad)
    assert bench.bytes_per_element(N, Npad) == pytest.approx(sum(stages) / 5, rel=1e-12)


def test_headline_bytes_per_launch():
    # 24^3 x 6 = 82,944 tets at N=5 (Np = 56, rows padded to 56 floats)
    assert bench.bytes_per_element(5, 56) == pytest.approx(5267.2, rel=1e-12)
    assert 82944 * bench.bytes_per_element(5, 56) == pytest.approx(436.8826368e6, rel=1e-12)
    # N=7: Np = 120
    assert bench.bytes_per_element(7, 120) == pytest.approx(11104.0, rel=1e-12)


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_flops_volume_term_dominates_as_stated(N):
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfp = (N + 1) * (N + 2) // 2
    f = bench.flops_per_element(N)
    volume = 36 * Np * Np        # three reference derivatives of six fields, multiply-add = 2 flops
    lift = 48 * Np * Nfp         # LIFT (Np x 4 Nfp) on six fields
    assert f >= volume + lift
    # the remaining terms (chain rule, curls, flux, update) are linear in Np and Nfp
    rest = f - volume - lift
    assert 0 < rest <= 100 * Np + 300 * Nfp
