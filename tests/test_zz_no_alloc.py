"""The allocation-free density entry point (elbm_density_noalloc), for
callers that may not allocate device memory, against the existing entry
points on the same state. Collected last so a stop at the first failure has
run every other test first; passes alone in a fresh process too."""
import ctypes
import math

import numpy as np
import pytest

from paper_1612_05404_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_density_noalloc_matches_step_moments_twice():
    import torch
    assert torch.cuda.is_available()
    from paper_1612_05404_gb300 import build, elbm
    build.build()
    torch.cuda.set_device(0)
    shape = (12, 10, 8)
    N = 960
    cfg = W.base_params(shape=shape, precision="fp64", store_macro=1,
                        face_bc=["periodic"] * 2 + ["wall"] * 4,
                        phi_bc=["periodic"] * 2 + ["neumann"] * 4)
    mask = np.zeros(N, np.uint8)
    mask[[14, 15, 300, 555, 700]] = W.SOLID
    rho0 = W.drop_profile(shape, 3.0) + W.uniform_noise(N, 1e-3, 7)
    sim = elbm.Sim(cfg, dict(mask=mask, rho=rho0))
    sim.step(2)
    stream = torch.cuda.current_stream()
    d_mask = torch.from_numpy(mask).cuda()
    for call in range(2):                     # two calls in a row on the shared scratch
        f_t = sim.get("f")                    # f(r, t) through the existing entry point
        sim.step(1)                           # its moments pass computes rho(t) from f(r, t)
        rho_ref = sim.get("rho")
        mass_ref = sim.diag()["mass"]
        d_f = torch.from_numpy(f_t).cuda()
        d_rho = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        d_mass = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = elbm.density_noalloc(d_f.data_ptr(), d_mask.data_ptr(), N, d_rho.data_ptr(),
                                  d_mass.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert rc == elbm.OK
        torch.cuda.synchronize()
        rho = d_rho.cpu().numpy()
        assert np.array_equal(rho, rho_ref), call
        assert d_mass.item() == pytest.approx(mass_ref, rel=1e-12), call
    # sizes beyond the fixed scratch are refused, nothing is launched
    big = elbm.NOALLOC_MAX_SITES + 1
    assert elbm.density_noalloc(d_f.data_ptr(), 0, big, d_rho.data_ptr(), d_mass.data_ptr()) == elbm.E_INVAL
    sim.close()


def test_density_noalloc_many_blocks_no_mask():
    """About 300k sites (293 blocks of partial sums, more than the 256
    threads of the final pass) with mask = NULL: rho bit for bit equal to
    the plane-by-plane sum p = 0..18 in FP64, and the mass to 1e-12 of the
    exactly rounded sum; two calls in a row."""
    import torch
    from paper_1612_05404_gb300 import build, elbm
    build.build()
    torch.cuda.set_device(0)
    N = 300_000
    f = W.random_populations(N, 0.05, 20161230)
    ref = f[0].copy()
    for p in range(1, 19):
        ref += f[p]
    d_f = torch.from_numpy(np.ascontiguousarray(f).reshape(-1)).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        d_rho = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        d_mass = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = elbm.density_noalloc(d_f.data_ptr(), 0, N, d_rho.data_ptr(), d_mass.data_ptr(),
                                  ctypes.c_void_p(stream.cuda_stream))
        assert rc == elbm.OK
        torch.cuda.synchronize()
        assert np.array_equal(d_rho.cpu().numpy(), ref), call
        assert d_mass.item() == pytest.approx(math.fsum(ref), rel=1e-12), call
