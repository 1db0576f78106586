"""dn_full_forward_noalloc: the full forward pass for callers that cannot
allocate device memory while they run (their device memory is reserved up
front, or allocation is forbidden after warm-up).  It must give the same
log-amplitudes as dn_full_forward, make no allocator call, and work on
consecutive calls that reuse its fixed scratch array.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import ModelDesc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dn():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_11189_gb300 import dysonnet
    lib = dysonnet._lib()
    fn = lib.dn_full_forward_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    return dysonnet


def _noalloc(dn, model, spins, prec):
    B, N = spins.shape
    lp = torch.empty(B, dtype=torch.float64, device="cuda")
    om = torch.empty((B, model.desc.dout), dtype=torch.float64, device="cuda")
    st = dn._lib().dn_full_forward_noalloc(model._h, N, ctypes.c_void_p(spins.data_ptr()), B,
                                           dn.PRECISIONS[prec], ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                           ctypes.c_void_p(lp.data_ptr()), ctypes.c_void_p(om.data_ptr()))
    return st, lp, om


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_noalloc_matches_full_forward_on_consecutive_calls(dn, prec, tol):
    cfg = synth.CONFIGS["lrtfim_n128"]
    model = dn.Model(cfg["desc"], synth.make_params(cfg))
    calls = {"alloc": 0}

    def alloc(n, stream):
        calls["alloc"] += 1
        return 0

    def free(p, n, stream):
        calls["alloc"] += 1

    # Two different batches back to back (the second reuses the scratch the first left behind).
    batches = [torch.from_numpy(synth.spins_uniform(24, 128, 7)).cuda(),
               torch.from_numpy(synth.spins_uniform(9, 128, 8)).cuda()]
    refs = [model.full_forward(s, prec=prec, with_omega=True) for s in batches]
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    dn.set_allocator(alloc, free)          # any allocation attempt would be counted (and refused)
    try:
        outs = [_noalloc(dn, model, s, prec) for s in batches]
        torch.cuda.synchronize()
    finally:
        dn.set_allocator(None, None)
        dn.install_torch_allocator()
    assert calls["alloc"] == 0
    for (st, lp, om), (lp_ref, om_ref) in zip(outs, refs):
        assert st == dn.DN_OK
        a, b = lp.cpu().numpy(), lp_ref.cpu().numpy()
        assert np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))) <= tol
        a, b = om.cpu().numpy(), om_ref.cpu().numpy()
        assert np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))) <= tol
    assert torch.cuda.memory_allocated() - before < (1 << 20)   # only the result tensors
    # The same amplitudes against the CPU FP64 oracle.
    for (st, lp, _), s in zip(outs, batches):
        lp_or, _ = oracle.logpsi(cfg["desc"], synth.make_params(cfg), s.cpu().numpy())
        assert np.max(np.abs(lp.cpu().numpy() - lp_or) / np.maximum(1.0, np.abs(lp_or))) <= tol
    model.close()


def test_noalloc_other_shapes_and_capacity(dn):
    desc = ModelDesc(L=3, d=5, s=3, w=1, dh=4, dout=2, periodic=1)
    params = synth.init_params(desc, 42, a_scale=5.0)
    model = dn.Model(desc, params)
    spins = torch.from_numpy(synth.spins_uniform(6, 11, 3)).cuda()
    st, lp, om = _noalloc(dn, model, spins, "fp64")
    lp_ref = model.full_forward(spins, prec="fp64")
    assert st == dn.DN_OK
    np.testing.assert_allclose(lp.cpu().numpy(), lp_ref.cpu().numpy(), rtol=1e-10, atol=1e-12)
    # A batch that does not fit the fixed scratch is refused without touching the outputs.
    big = torch.ones((4096, 128), dtype=torch.int8, device="cuda")
    cfg = synth.CONFIGS["lrtfim_n128"]
    model2 = dn.Model(cfg["desc"], synth.make_params(cfg))
    st, _, _ = _noalloc(dn, model2, big, "fp32")
    assert st == dn.DN_EINVAL
    model.close()
    model2.close()
