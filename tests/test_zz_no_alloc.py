"""The allocation-free residual entry point (snac_residual_noalloc).

It serves callers that cannot allocate device memory -- programs whose device memory belongs to
their own caching allocator or to a fixed budget, and tight loops that cannot pay for the
device-wide synchronisation of cudaMalloc/cudaFree -- and therefore cannot create a plan. Its
scratch is a fixed device array shared by every call. These tests call it through the C ABI and
check it against the plan-based snac_residual (same tolerance as the other stage tests), on two calls
in a row with different problems so that state left in the shared scratch by the first call cannot
leak into the second. This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2106_03583_gb300 import inputs, snac

from gpu_util import dev, host, plan, rel

pytestmark = pytest.mark.gpu


def _one_block(nx, ny, nz, walls, zbc, stretched, periodic=(False, False)):
    xf = inputs.tanh_faces(nx, 0, 1.4 if stretched else 0.0, 0.0, 1.5)
    yf = inputs.tanh_faces(ny, 1, 1.1 if stretched else 0.0, 0.0, 1.0)
    zf = np.linspace(0.0, 0.7, nz + 1)
    wb = {"x-": walls[0], "x+": walls[1], "y-": walls[2], "y+": walls[3]}
    return inputs.make_blocks(xf, yf, zf, [(0, nx, 0, ny)], wb, zbc, periodic=periodic)[0]


CASES = [
    ((96, 72, 32, ("D", "D", "N", "N"), ("P", "P"), True, (False, False)),
     (40, 24, 10, ("N", "D", "D", "N"), ("N", "D"), True, (False, False))),
    ((72, 36, 18, ("N", "N", "N", "N"), ("N", "N"), False, (True, True)),
     (128, 64, 64, ("D", "N", "N", "D"), ("D", "D"), True, (False, False))),
]


@pytest.mark.parametrize("first,second", CASES)
def test_noalloc_residual_matches_plan_residual_twice(first, second):
    import torch
    for k, (nx, ny, nz, walls, zbc, st, per) in enumerate((first, second)):
        block = _one_block(nx, ny, nz, walls, zbc, st, per)
        n = nx * ny * nz
        rng = np.random.default_rng(10 + k)
        f, p = dev(rng.standard_normal(n)), dev(rng.standard_normal(n))
        r_na = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        r2_na, f2_na = snac.residual_noalloc(block, f, p, r_na)
        pl = plan([block])
        r_pl = torch.empty_like(r_na)
        r2_pl, f2_pl = pl.residual(f, p, r_pl)
        pl.close()
        assert rel(host(r_na), host(r_pl)) <= 1e-13
        assert abs(r2_na - r2_pl) <= 1e-12 * r2_pl
        assert abs(f2_na - f2_pl) <= 1e-12 * f2_pl


def test_noalloc_rejects_what_its_scratch_cannot_hold():
    import torch
    n_big = 4097
    big = _one_block(n_big, 8, 2, ("D", "D", "N", "N"), ("P", "P"), False)
    n = n_big * 8 * 2
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(snac.SnacError) as e:
        snac.residual_noalloc(big, t, t, torch.empty_like(t))
    assert e.value.name == "INVALID_ARG" and "4096" in str(e.value)
    two = inputs.make_blocks(np.linspace(0, 1, 9), np.linspace(0, 1, 5), np.linspace(0, 1, 3),
                             [(0, 4, 0, 4), (4, 8, 0, 4)], {"x-": "D", "x+": "D", "y-": "N", "y+": "N"},
                             ("P", "P"))
    t = torch.zeros(4 * 4 * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(snac.SnacError) as e:
        snac.residual_noalloc(two[0], t, t, torch.empty_like(t))
    assert e.value.name == "INVALID_ARG"
