"""Serving loop (dn_server_*): requests for chains of different N, batched together,
against the FP64 oracle and against the same requests served one at a time.

A request's ratios must not depend on the other requests of its batch: every flip is
evaluated by its own CTA from its own chain's cache, so the results served alone and
in the mix are compared for equality; both are compared with the oracle at the
precision's bound (1e-10 FP64, 1e-4 FP32, the rel metric of the parity tests).
"""
import numpy as np
import pytest
import torch  # noqa: F401  (CUDA context for the library)

import oracle
import synth
from synth import ModelDesc

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}


@pytest.fixture(scope="module")
def dn():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_11189_gb300 import dysonnet
    return dysonnet


def rel_err(got, ref, lp_ref):
    den = np.maximum(np.abs(ref), 1e-3 * (1.0 + abs(lp_ref)))
    return np.abs(got - ref) / den


def make_requests(chain_N, n_req, max_f, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n_req):
        c = int(rng.integers(len(chain_N)))
        F = int(rng.integers(1, max_f + 1))
        reqs.append((c, rng.integers(0, chain_N[c], size=F).astype(np.int32)))
    return reqs


def serve(dn, model, prec, mode, chains, reqs, budget=8 << 30, alone=False):
    srv = dn.Server(model, prec=prec, mode=mode, hbm_budget_bytes=budget, max_batch_flips=256, max_batch_chains=8)
    for c, sp in enumerate(chains):
        srv.set_chain(c, sp)
    out = []
    if alone:
        for c, sites in reqs:
            out.append(srv.wait(srv.submit(c, sites), timeout_s=120.0)[0])
    else:
        tickets = [srv.submit(c, sites) for c, sites in reqs]
        out = [srv.wait(t, timeout_s=120.0)[0] for t in tickets]
    stats = srv.stats()
    srv.close()
    return out, stats


def check_oracle(desc, params, chains, reqs, out, tol):
    lp = [oracle.logpsi(desc, params, sp[None, :])[0][0] for sp in chains]
    for (c, sites), got in zip(reqs, out):
        F = len(sites)
        sites2 = np.stack([sites, -np.ones(F, dtype=np.int32)], axis=1)
        ref = oracle.dlogpsi(desc, params, chains[c][None, :], np.zeros(F, dtype=np.int32), sites2)
        e = rel_err(got, ref, lp[c]).max()
        assert e <= tol, f"chain {c}: max rel err {e:.3e}"


def setup_model(desc, seed, chain_N):
    params = synth.init_params(desc, seed, a_scale=6.0)
    chains = [synth.spins_uniform(1, N, 50 + N)[0] for N in chain_N]
    return params, chains


@pytest.mark.parametrize("mode", ["abacus", "persistent"])
def test_serving_mixed_equals_alone_and_oracle_fp64(dn, mode):
    desc = ModelDesc(L=3, d=8, s=4, w=1, dh=8, dout=2, periodic=0)
    chain_N = [12, 17, 24, 31]
    params, chains = setup_model(desc, 301, chain_N)
    reqs = make_requests(chain_N, 24, 10, seed=1)
    model = dn.Model(desc, params)
    mixed, st = serve(dn, model, "fp64", mode, chains, reqs)
    alone, st1 = serve(dn, model, "fp64", mode, chains, reqs, alone=True)
    model.close()
    assert st["requests"] == len(reqs) and st["flips"] == sum(len(s) for _, s in reqs)
    assert st["batches"] >= 1 and st1["batches"] == len(reqs)
    for a, b in zip(mixed, alone):
        assert np.array_equal(a, b)
    check_oracle(desc, params, chains, reqs, mixed, TOL["fp64"])


@pytest.mark.parametrize("mode", ["abacus", "persistent"])
def test_serving_budget_evicts_and_stays_exact(dn, mode):
    desc = ModelDesc(L=3, d=8, s=4, w=1, dh=8, dout=2, periodic=1)
    chain_N = [15, 22, 30]
    params, chains = setup_model(desc, 302, chain_N)
    model = dn.Model(desc, params)
    one = max(model.cache_bytes(N, 1, "fp64") for N in chain_N)
    reqs = make_requests(chain_N, 18, 6, seed=2)
    out, st = serve(dn, model, "fp64", mode, chains, reqs, budget=int(1.5 * one))
    model.close()
    assert st["evictions"] > 0
    assert st["resident_bytes"] <= int(1.5 * one)
    check_oracle(desc, params, chains, reqs, out, TOL["fp64"])


def test_serving_recompute_mode_fp64(dn):
    desc = ModelDesc(L=2, d=6, s=3, w=1, dh=6, dout=2, periodic=0)
    chain_N = [9, 14]
    params, chains = setup_model(desc, 303, chain_N)
    reqs = make_requests(chain_N, 8, 7, seed=3)
    model = dn.Model(desc, params)
    out, st = serve(dn, model, "fp64", "recompute", chains, reqs)
    model.close()
    assert st["cache_builds"] == 0
    check_oracle(desc, params, chains, reqs, out, TOL["fp64"])


def test_serving_fp32_d64_chains(dn):
    desc = ModelDesc(L=4, d=64, s=8, w=2, dh=32, dout=2, periodic=0)
    chain_N = [40, 70, 33]
    params, chains = setup_model(desc, 304, chain_N)
    reqs = make_requests(chain_N, 12, 40, seed=4)
    model = dn.Model(desc, params)
    mixed, _ = serve(dn, model, "fp32", "abacus", chains, reqs)
    alone, _ = serve(dn, model, "fp32", "abacus", chains, reqs, alone=True)
    resident, _ = serve(dn, model, "fp32", "persistent", chains, reqs)
    model.close()
    for a, b, c in zip(mixed, alone, resident):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    check_oracle(desc, params, chains, reqs, mixed, TOL["fp32"])


def test_serving_rejects_bad_requests(dn):
    desc = ModelDesc(L=2, d=4, s=3, w=1, dh=4, dout=2, periodic=0)
    params = synth.init_params(desc, 5, a_scale=2.0)
    model = dn.Model(desc, params)
    srv = dn.Server(model, prec="fp64", max_batch_flips=16)
    with pytest.raises(dn.DysonNetError):
        srv.set_chain(0, np.array([1, 0, -1], dtype=np.int8))
    srv.set_chain(0, np.array([1, -1, 1, 1, -1], dtype=np.int8))
    with pytest.raises(dn.DysonNetError):
        srv.submit(3, np.array([0], dtype=np.int32))          # unknown chain
    with pytest.raises(dn.DysonNetError):
        srv.submit(0, np.zeros(17, dtype=np.int32))           # larger than a batch
    t = srv.submit(0, np.array([0, 4], dtype=np.int32))
    r, lat = srv.wait(t, timeout_s=60.0)
    assert r.shape == (2,) and np.all(np.isfinite(r)) and lat >= 0.0
    srv.close()
    model.close()


def test_persistent_kernel_waits_are_bounded(dn):
    """The resident kernel of a persistent server waits for work only up to its idle
    limit: with the queue left unfed it leaves and reports DN_ETIMEOUT, and the next
    request launches it again and is served exactly."""
    desc = ModelDesc(L=3, d=8, s=4, w=1, dh=8, dout=2, periodic=0)
    chain_N = [13, 21]
    params, chains = setup_model(desc, 305, chain_N)
    model = dn.Model(desc, params)
    srv = dn.Server(model, prec="fp64", mode="persistent", max_batch_flips=64)
    st, running = srv.kernel_status()
    assert st == dn.DN_OK and not running               # nothing launched yet
    srv.set_idle_limit(0.05)
    for c, sp in enumerate(chains):
        srv.set_chain(c, sp, build_now=True)
    reqs = make_requests(chain_N, 6, 8, seed=5)
    out = [srv.wait(srv.submit(c, sites), timeout_s=60.0)[0] for c, sites in reqs]
    st, running = srv.kernel_status(wait_s=5.0)         # no more work: the idle limit runs out
    assert st == dn.DN_ETIMEOUT and not running
    more = make_requests(chain_N, 4, 8, seed=6)
    out += [srv.wait(srv.submit(c, sites), timeout_s=60.0)[0] for c, sites in more]
    st, running = srv.kernel_status(wait_s=5.0)
    assert st == dn.DN_ETIMEOUT and not running
    srv.close()
    model.close()
    check_oracle(desc, params, chains, reqs + more, out, TOL["fp64"])


def test_persistent_relaunch_while_requests_arrive(dn):
    """A persistent server whose idle limit (2 ms) is about as long as the gaps between
    requests: the kernel leaves and is launched again while requests are in flight, so
    items published after some CTAs left are served by the next launch and items the
    previous launch served are dropped by their state words.  Every request completes
    exactly once with the oracle's ratios and the batch server's values."""
    import time
    desc = ModelDesc(L=3, d=8, s=4, w=1, dh=8, dout=2, periodic=0)
    chain_N = [12, 19, 26]
    params, chains = setup_model(desc, 307, chain_N)
    reqs = make_requests(chain_N, 48, 40, seed=7)
    gaps = np.random.default_rng(8).uniform(0.0, 0.006, size=len(reqs))
    model = dn.Model(desc, params)
    srv = dn.Server(model, prec="fp64", mode="persistent", max_batch_flips=64)
    srv.set_idle_limit(0.002)
    for c, sp in enumerate(chains):
        srv.set_chain(c, sp, build_now=True)
    tickets = []
    for (c, sites), gap in zip(reqs, gaps):
        tickets.append(srv.submit(c, sites))
        time.sleep(gap)
    out = [srv.wait(t, timeout_s=60.0)[0] for t in tickets]
    st, running = srv.kernel_status(wait_s=5.0)
    assert st == dn.DN_ETIMEOUT and not running
    srv.close()
    ref, _ = serve(dn, model, "fp64", "abacus", chains, reqs)
    model.close()
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)
    check_oracle(desc, params, chains, reqs, out, TOL["fp64"])


def test_persistent_mode_rejected_options(dn):
    desc = ModelDesc(L=2, d=4, s=3, w=1, dh=4, dout=2, periodic=0)
    model = dn.Model(desc, synth.init_params(desc, 6, a_scale=2.0))
    srv = dn.Server(model, prec="fp64", mode="abacus", max_batch_flips=16)
    with pytest.raises(dn.DysonNetError):
        srv.set_idle_limit(0.1)                          # only persistent servers have a resident kernel
    assert srv.kernel_status()[0] == dn.DN_EINVAL
    srv.close()
    srv = dn.Server(model, prec="fp64", mode="persistent", max_batch_flips=16)
    with pytest.raises(dn.DysonNetError):
        srv.set_idle_limit(0.0)
    srv.close()
    model.close()
