"""The C-ABI library builds, loads without a GPU, exports every entry point
declared in include/elbm.h, and its ctypes mirror has the C layout."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_1612_05404_gb300 import build as B
from paper_1612_05404_gb300 import elbm
from paper_1612_05404_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return elbm.lib()


def test_exports_every_declared_symbol(L):
    hdr = open(os.path.join(ROOT, "include", "elbm.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"^\s*(?:const\s+)?(?:\w+\s+)*\w+\s*\**\s*(elbm_[a-z_0-9]+)\s*\(", hdr, re.M))
    assert declared >= set(elbm.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", elbm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (elbm_[a-z_]+)$", out, re.M))
    assert declared <= exported, declared - exported
    for name in declared:
        assert getattr(L, name)


def test_velocity_sets_link_side_by_side(L):
    """The step's kernels are compiled once per velocity set into one
    library (D3Q19, and the paper's D2Q9 in k_*_d2q9.cu) under distinct
    names, so that a launch for one set can never reach the other's code;
    the D2Q9 build holds only the variants elbm_init accepts for it (no BF16
    storage, no learned proposal)."""
    out = subprocess.run(["nm", "-C", elbm.LIB_PATH], capture_output=True, text=True, check=True).stdout
    for ns in ("elbm::d3q19::", "elbm::d2q9::"):
        for k in ("k_collide<", "k_moments<", "k_charge_ab<", "k_sor<", "k_init_pop<", "k_bounce_bits("):
            assert ns + k in out, ns + k
    assert "elbm::d3q19::k_collide<2," in out and "elbm::d3q19::k_collide<1, 1, true>" in out
    assert "elbm::d2q9::k_collide<2," not in out and "elbm::d2q9::k_collide<1, 1, true>" not in out
    assert "elbm::d2q9::k_mg_" not in out  # multigrid is shared and D3Q19-instantiated only


def test_struct_layout_matches_c(L):
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "elbm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(elbm_params), offsetof(elbm_params, phi_lo),
         offsetof(elbm_params, nu0), offsetof(elbm_params, E_ext), offsetof(elbm_params, rho_out),
         offsetof(elbm_params, cuda_stream), sizeof(elbm_init_fields));
  printf("%zu\n", offsetof(elbm_params, velset));
  return 0; }
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        got = list(map(int, subprocess.run([exe], capture_output=True, text=True).stdout.split()))
    P = elbm.Params
    want = [ctypes.sizeof(P), P.phi_lo.offset, P.nu0.offset, P.E_ext.offset, P.rho_out.offset,
            P.cuda_stream.offset, ctypes.sizeof(elbm.InitFields), P.velset.offset]
    assert got == want


def test_velocity_set_matches_oracle_table(L):
    c, w = elbm.velocity_set()
    co, wo, _ = oracle.lattice(3)
    assert np.array_equal(c, co) and np.array_equal(w, wo)


def test_d2q9_velocity_set_matches_oracle_table(L):
    """The CUDA path's D2Q9 order and weights (Sec. II) are the oracle's."""
    c, w = elbm.velocity_set(2)
    co, wo, _ = oracle.lattice(2)
    assert c.shape == (9, 3) and np.array_equal(c, co) and np.array_equal(w, wo)
    assert L.elbm_velocity_set_of(7, None, None) == elbm.E_INVAL


def test_strerror(L):
    assert elbm.strerror(0) == "ok"
    assert "invalid" in elbm.strerror(-1)


@pytest.mark.parametrize("bad", [
    dict(shape=(0, 4, 4)),
    dict(face_bc=["wall", "periodic", "periodic", "periodic", "periodic", "periodic"]),
    dict(phi_bc=["dirichlet"] * 2 + ["periodic"] * 4),
    dict(nu0=0.0),
    dict(charge_model="transport", poisson_solver="mg", shape=(3, 4, 4)),  # no multigrid level
    dict(precision="fp16"),
    dict(carreau_lagged=2),
    dict(alpha_h_tol=-1e-10),
    dict(alpha_h_tol=float("nan")),
    # D2Q9: one site thick, in-plane potential data, and the kernels it is built for
    dict(dim=2),                                                  # nz = 4
    dict(dim=2, shape=(4, 4, 1), precision="bf16"),
    dict(dim=2, shape=(4, 4, 1), precision="fp32", alpha_precision="fp32_fast"),
    dict(dim=2, shape=(4, 4, 1), charge_model="transport"),
    dict(dim=2, shape=(4, 4, 1), charge_model="conserved", poisson_solver="mg"),
    dict(dim=2, shape=(4, 4, 1), phi_axis=2),
    dict(dim=2, shape=(4, 4, 1), E_ext=(0.0, 0.0, 1e-3)),
    dict(dim=4, shape=(4, 4, 1)),                                 # no such set
])
def test_invalid_parameters_rejected_without_allocation(L, bad):
    cfg = W.base_params(shape=(4, 4, 4))
    try:
        cfg.update(bad)
        P = elbm.make_params(cfg)
    except KeyError:
        return  # not even representable
    N = int(np.prod(cfg["shape"])) if min(cfg["shape"]) > 0 else 1
    rho = np.ones(max(N, 1))
    IF = elbm.InitFields()
    IF.rho0 = rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    assert L.elbm_init(ctypes.byref(P), ctypes.byref(IF), 1, ctypes.byref(h)) == elbm.E_INVAL
    assert not h.value


def test_null_arguments(L):
    assert L.elbm_init(None, None, 1, None) == elbm.E_INVAL
    assert L.elbm_step(None, 1) == elbm.E_INVAL
    L.elbm_free(None)


def test_alpha_eval_argument_checks(L):
    """elbm_alpha_eval validates before touching the device: bad arguments
    return ELBM_E_INVAL and n = 0 enqueues nothing (both run without a GPU)."""
    import ctypes
    p = ctypes.c_void_p(16)  # never dereferenced: every call below fails validation or has n = 0
    assert L.elbm_alpha_eval(None, 0, 1, 1e-5, None, None, None, None, None, None) == 0
    assert L.elbm_alpha_eval(p, -1, 1, 1e-5, None, p, None, None, None, None) == elbm.E_INVAL
    assert L.elbm_alpha_eval(None, 5, 1, 1e-5, None, p, None, None, None, None) == elbm.E_INVAL
    assert L.elbm_alpha_eval(p, 5, 1, 1e-5, None, None, None, None, None, None) == elbm.E_INVAL
    assert L.elbm_alpha_eval(p, 5, 7, 1e-5, None, p, None, None, None, None) == elbm.E_INVAL
    assert L.elbm_alpha_eval(p, 5, 1, 1e-9, None, p, None, None, None, None) == elbm.E_INVAL
    assert L.elbm_alpha_eval(p, 5, 1, -1.0, None, p, None, None, None, None) == elbm.E_INVAL
    assert L.elbm_alpha_eval(p, 5, 0, 1e-5, p, p, None, None, None, None) == elbm.E_INVAL  # learned needs FP32


def test_mlp_entry_points_argument_checks(L):
    """Validation before any launch (runs without a GPU; no call below reaches
    a kernel)."""
    import ctypes
    p = ctypes.c_void_p(16)
    assert L.elbm_mlp_workspace_floats(0) == 0
    assert L.elbm_mlp_workspace_floats(128) == 2 * 5570
    assert L.elbm_alpha_features(None, 0, None, None, None) == 0
    assert L.elbm_alpha_features(p, -2, p, None, None) == elbm.E_INVAL
    assert L.elbm_alpha_features(p, 3, None, None, None) == elbm.E_INVAL
    assert L.elbm_alpha_harvest(p, 3, 1e-9, p, p, p, None) == elbm.E_INVAL
    assert L.elbm_alpha_harvest(p, 3, 1e-5, p, p, None, None) == elbm.E_INVAL
    assert L.elbm_mlp_forward(p, 3, p, 5, p, None) == elbm.E_INVAL
    assert L.elbm_mlp_forward(p, 3, None, 1, p, None) == elbm.E_INVAL
    assert L.elbm_mlp_grad(p, p, 0, p, p, None, p, None) == elbm.E_INVAL
    assert L.elbm_mlp_grad(p, p, 4, p, p, None, None, None) == elbm.E_INVAL
    assert L.elbm_mlp_adam(p, p, p, p, 0, 1e-3, 0.9, 0.999, 1e-8, None) == elbm.E_INVAL
    assert L.elbm_mlp_adam(p, p, p, p, 1, 1e-3, 1.0, 0.999, 1e-8, None) == elbm.E_INVAL
    assert L.elbm_mlp_train(p, p, 4, p, p, p, 0, 1, 8, 1e-3, 0, None, p, None) == elbm.E_INVAL
    assert L.elbm_mlp_train(p, p, 4, p, p, p, 0, 1, 0, 1e-3, 1, None, p, None) == elbm.E_INVAL


def test_batch_create_argument_checks(L):
    import ctypes
    out = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 1)(None)
    assert L.elbm_batch_create(arr, 1, 0, None, None) == elbm.E_INVAL
    assert L.elbm_batch_create(None, 1, 0, None, ctypes.byref(out)) == elbm.E_INVAL
    assert L.elbm_batch_create(arr, 0, 0, None, ctypes.byref(out)) == elbm.E_INVAL
    assert L.elbm_batch_create(arr, 1, 0, None, ctypes.byref(out)) == elbm.E_INVAL  # a NULL instance
    assert L.elbm_batch_create(arr, 1, 6, None, ctypes.byref(out)) == elbm.E_INVAL  # unknown flag
    assert L.elbm_batch_create(arr, 1, 17 << 8, None, ctypes.byref(out)) == elbm.E_INVAL  # span above 16
    assert not out.value


def test_paper_2d_workloads_pass_the_host_checks(L):
    """The paper's 2-D runs on D2Q9 (the drop at rest and in a field, the jet
    cases a/b/c with the adaptive inlet, FP64 and FP32): elbm_init's host
    checks accept each, inlet region and all; only the device allocation can
    then fail (no GPU here)."""
    runs = [W.paper_drop_2d(n=40, radius=8.0)]
    cfg, fl = W.paper_drop_2d(n=40, radius=8.0)
    cfg.update(E_ext=(0.5, 0.0, 0.0), force_el="full", precision="fp32", alpha_precision="fp32")
    W.reduced_precision(cfg)
    runs.append((cfg, fl))
    for case in "abc":
        for prec in ("fp64", "fp32"):
            runs.append(W.jet_2d(n=48, D=12, nozzle_len=10, wall=2, case=case, precision=prec))
    for cfg, fl in runs:
        try:
            elbm.Sim(cfg, fl).close()
        except elbm.ElbmError as e:
            assert e.code != elbm.E_INVAL, (cfg["charge_model"], cfg["precision"], e)


def test_every_box_edge_passes_the_multigrid_checks(L):
    """The batched-droplet boxes (periodic, FP32, multigrid) of every integer
    edge 24..96, odd ones included: elbm_init's host checks (parameters, the
    multigrid hierarchy with odd extents coarsened to (n + 1)/2 cells, the
    one-CTA tail of at most 4096 cells) accept each; only the device
    allocation can then fail (no GPU here). A lattice whose extents cannot
    coarsen at all is refused before that."""
    for edge in W.BATCH_EDGES:
        cfg, fields = W.batched_droplet(edge, 5e-4, 0.7, precision="fp32")
        P = elbm.make_params(cfg)
        IF = elbm.InitFields()
        rho = np.ascontiguousarray(fields["rho"], dtype=np.float64)
        IF.rho0 = rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        rc = L.elbm_init(ctypes.byref(P), ctypes.byref(IF), 1, ctypes.byref(h))
        assert rc != elbm.E_INVAL, edge
        if h.value:
            L.elbm_free(h)
    cfg = W.base_params(shape=(3, 4, 4), charge_model="transport", poisson_solver="mg", precision="fp32",
                        alpha_eq_tol=1e-5)
    P = elbm.make_params(cfg)
    IF = elbm.InitFields()
    rho = np.ones(48)
    IF.rho0 = rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    assert L.elbm_init(ctypes.byref(P), ctypes.byref(IF), 1, ctypes.byref(h)) == elbm.E_INVAL
    assert not h.value
