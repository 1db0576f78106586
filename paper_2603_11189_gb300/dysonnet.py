"""Thin Python binding of libdysonnet.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module converts
torch tensors to raw pointers and status codes to exceptions.  It raises if
the library is missing or no CUDA device is present: there is no CPU path.

Names follow the C ABI in include/dysonnet.h.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

DN_OK, DN_EINVAL, DN_ENOMEM, DN_ECUDA, DN_ETIMEOUT, DN_EUNSUPPORTED = range(6)
DN_FP64, DN_FP32, DN_BF16 = 0, 1, 2
PRECISIONS = {"fp64": DN_FP64, "fp32": DN_FP32, "bf16": DN_BF16,
              torch.float64: DN_FP64, torch.float32: DN_FP32, torch.bfloat16: DN_BF16}


class DysonNetError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_lib().dn_status_string(status).decode()}")


class ModelDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("L", "d", "s", "w", "d_h", "d_out", "periodic", "f_kind")]


class Hamiltonian(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("J", ctypes.c_double), ("alpha", ctypes.c_double), ("h", ctypes.c_double),
                ("J1", ctypes.c_double), ("J2", ctypes.c_double), ("periodic", ctypes.c_int), ("kac", ctypes.c_int)]


class SamplerStats(ctypes.Structure):
    _fields_ = [("proposals", ctypes.c_ulonglong), ("accepted", ctypes.c_ulonglong), ("refreshes", ctypes.c_ulonglong)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_ulonglong), ("flips", ctypes.c_ulonglong), ("batches", ctypes.c_ulonglong),
                ("cache_builds", ctypes.c_ulonglong), ("evictions", ctypes.c_ulonglong),
                ("resident_bytes", ctypes.c_size_t)]


DN_SERVE_ABACUS, DN_SERVE_RECOMPUTE, DN_SERVE_PERSISTENT = 0, 1, 2

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_L = None
_torch_alloc_installed = False
_keep = []


def library_path() -> str:
    return _build.LIB


def _lib():
    global _L
    if _L is not None:
        return _L
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libdysonnet.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i32, sz, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
    sig = {
        "dn_status_string": (ctypes.c_char_p, [i32]),
        "dn_set_allocator": (i32, [ALLOC_FN, FREE_FN, vp]),
        "dn_model_create": (i32, [ctypes.POINTER(ModelDesc), vp, sz, ctypes.POINTER(vp)]),
        "dn_model_destroy": (None, [vp]),
        "dn_cache_bytes": (sz, [vp, i32, i32, i32, i32]),
        "dysonnet_forward_cache": (i32, [vp, i32, vp, i32, i32, i32, vp, ctypes.POINTER(vp), vp]),
        "abacus_flip_ratios": (i32, [vp, vp, vp, i32, vp, vp]),
        "abacus_single_flip_ratios": (i32, [vp, vp, vp]),
        "abacus_pair_flip_ratios": (i32, [vp, i32, ctypes.POINTER(ctypes.c_int32), vp, vp]),
        "local_energy": (i32, [vp, ctypes.POINTER(Hamiltonian), i32, vp, i32, i32, vp, vp]),
        "dn_full_forward": (i32, [vp, i32, vp, i32, i32, vp, vp, vp]),
        "dn_recompute_flip_ratios": (i32, [vp, i32, vp, i32, vp, vp, i32, i32, vp, vp]),
        "dn_cache_check": (i32, [vp, vp]),
        "dn_cache_info": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                ctypes.POINTER(i32)]),
        "dn_cache_tensor": (i32, [vp, ctypes.c_char_p, ctypes.POINTER(vp), ctypes.POINTER(sz),
                                  ctypes.POINTER(i32)]),
        "dn_cache_destroy": (None, [vp]),
        "dn_server_create": (i32, [vp, i32, i32, sz, i32, i32, ctypes.POINTER(vp)]),
        "dn_server_set_chain": (i32, [vp, i32, i32, vp, i32]),
        "dn_server_submit": (i32, [vp, i32, vp, i32, vp, ctypes.POINTER(ctypes.c_ulonglong)]),
        "dn_server_wait": (i32, [vp, ctypes.c_ulonglong, dbl, ctypes.POINTER(dbl)]),
        "dn_server_get_stats": (i32, [vp, ctypes.POINTER(ServerStats)]),
        "dn_server_destroy": (None, [vp]),
        "dn_model_nparams": (sz, [vp]),
        "dn_logpsi_grad": (i32, [vp, i32, vp, i32, i32, vp, vp, vp, vp, vp]),
        "dn_sr_matrices": (i32, [vp, i32, sz, i32, vp, vp, sz, i32, vp]),
        "dn_sampler_batch": (i32, [vp, i32, vp, i32, vp, vp, i32, dbl, i32, vp, vp, ctypes.POINTER(SamplerStats)]),
        "dn_set_fused_links": (i32, [i32]),
        "dn_set_fft_links": (i32, [i32]),
        "dn_set_fft_conv": (i32, [i32]),
        "dn_server_set_idle_limit": (i32, [vp, dbl]),
        "dn_server_kernel_status": (i32, [vp, dbl, ctypes.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _L = L
    return L


def exported_symbols():
    """Names the binding expects from the library (all declared in dysonnet.h)."""
    return ["dn_status_string", "dn_set_allocator", "dn_model_create", "dn_model_destroy", "dn_cache_bytes",
            "dysonnet_forward_cache", "abacus_flip_ratios", "local_energy", "dn_full_forward",
            "dn_recompute_flip_ratios", "dn_cache_check", "dn_cache_info", "dn_cache_tensor", "dn_cache_destroy",
            "dn_full_forward_noalloc", "abacus_single_flip_ratios", "abacus_pair_flip_ratios", "dn_launch_count", "dn_profile_enable",
            "dn_profile_count", "dn_profile_get", "dn_server_create", "dn_server_set_chain", "dn_server_submit",
            "dn_server_wait", "dn_server_get_stats", "dn_server_destroy", "dn_model_nparams", "dn_logpsi_grad", "dn_sr_matrices", "dn_sampler_batch",
            "dn_set_fused_links", "dn_set_fft_links", "dn_set_fft_conv", "dn_server_set_idle_limit",
            "dn_server_kernel_status"]


def set_fused_links(on: bool):
    """Fused (default) or two-kernel end of the link-propagation chains; both exact."""
    _check(_lib().dn_set_fused_links(int(bool(on))), "dn_set_fused_links")


def set_fft_links(mode: int):
    """Band links of one-intermediate pairs: 0 direct sum, 1 FFT where it is the faster one
    (default), 2 FFT wherever the shape allows; all exact."""
    _check(_lib().dn_set_fft_links(int(mode)), "dn_set_fft_links")


def set_fft_conv(mode: int):
    """S4 convolution of the forward pass: 0 direct sum, 1 FFT for FP32 with N >= 512
    (default), 2 FFT wherever it applies; all exact to rounding."""
    _check(_lib().dn_set_fft_conv(int(mode)), "dn_set_fft_conv")


def _check(status: int, what: str):
    if status != DN_OK:
        raise DysonNetError(status, what)


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def install_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_alloc_installed
    if _torch_alloc_installed:
        return

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _keep.extend([a, f])
    _check(_lib().dn_set_allocator(a, f, None), "dn_set_allocator")
    _torch_alloc_installed = True


def set_allocator(alloc_py, free_py):
    """Install Python allocation callbacks (alloc(nbytes, stream) -> ptr or 0;
    free(ptr, nbytes, stream)); pass None, None for the library default."""
    global _torch_alloc_installed
    if alloc_py is None:
        _check(_lib().dn_set_allocator(ALLOC_FN(), FREE_FN(), None), "dn_set_allocator")
        _torch_alloc_installed = False
        return
    a = ALLOC_FN(lambda n, s, c: alloc_py(int(n), int(s or 0)) or None)
    f = FREE_FN(lambda p, n, s, c: free_py(int(p), int(n), int(s or 0)))
    _keep.extend([a, f])
    _check(_lib().dn_set_allocator(a, f, None), "dn_set_allocator")
    _torch_alloc_installed = False


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("the DysonNet library needs a CUDA device; there is no CPU fallback")


class Model:
    """A DysonNet model held by the library (weights copied at creation)."""

    def __init__(self, desc, params: np.ndarray, use_torch_allocator: bool = True):
        _require_cuda()
        if use_torch_allocator:
            install_torch_allocator()
        self.desc = desc
        self._d = ModelDesc(desc.L, desc.d, desc.s, desc.w, desc.dh, desc.dout, desc.periodic, desc.fkind)
        p = np.ascontiguousarray(params, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(_lib().dn_model_create(ctypes.byref(self._d), p.ctypes.data_as(ctypes.c_void_p), p.size,
                                      ctypes.byref(h)), "dn_model_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().dn_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cache_bytes(self, N: int, batch: int, prec="fp32", max_cluster: int = 1) -> int:
        return int(_lib().dn_cache_bytes(self._h, N, batch, PRECISIONS[prec], max_cluster))

    def forward_cache(self, spins: torch.Tensor, prec="fp32", max_cluster: int = 1, stream=None,
                      logpsi: torch.Tensor | None = None) -> "Cache":
        """dysonnet_forward_cache: spins int8 [B][N] on the device."""
        B, N = spins.shape
        h = ctypes.c_void_p()
        _check(_lib().dysonnet_forward_cache(self._h, N, _ptr(spins), B, PRECISIONS[prec], max_cluster,
                                             _stream(stream), ctypes.byref(h), _ptr(logpsi)),
               "dysonnet_forward_cache")
        return Cache(self, h, spins)

    def local_energy(self, ham: dict, spins: torch.Tensor, prec="fp32", stream=None,
                     out: torch.Tensor | None = None) -> torch.Tensor:
        B, N = spins.shape
        if out is None:
            out = torch.empty(B, dtype=torch.float64, device=spins.device)
        H = Hamiltonian(int(ham.get("kind", 0)), float(ham.get("J", 0.0)), float(ham.get("alpha", 0.0)),
                        float(ham.get("h", 0.0)), float(ham.get("J1", 0.0)), float(ham.get("J2", 0.0)),
                        int(ham.get("periodic", 0)), int(ham.get("kac", 0)))
        _check(_lib().local_energy(self._h, ctypes.byref(H), N, _ptr(spins), B, PRECISIONS[prec], _stream(stream),
                                   _ptr(out)), "local_energy")
        return out

    def full_forward(self, spins: torch.Tensor, prec="fp32", stream=None, with_omega=False):
        B, N = spins.shape
        lp = torch.empty(B, dtype=torch.float64, device=spins.device)
        om = torch.empty((B, self.desc.dout), dtype=torch.float64, device=spins.device) if with_omega else None
        _check(_lib().dn_full_forward(self._h, N, _ptr(spins), B, PRECISIONS[prec], _stream(stream), _ptr(lp),
                                      _ptr(om)), "dn_full_forward")
        return (lp, om) if with_omega else lp

    @property
    def nparams(self) -> int:
        return int(_lib().dn_model_nparams(self._h))

    def logpsi_grad(self, spins: torch.Tensor, prec="fp32", stream=None, weights: torch.Tensor | None = None,
                    with_O: bool = True):
        """(log psi [B] f64, O [B][nparams] or None, vjp [nparams] f64 or None): the per-configuration
        log-derivatives d log psi / d theta and, with `weights` [B] f64, sum_b w_b O_b."""
        B, N = spins.shape
        dev = spins.device
        lp = torch.empty(B, dtype=torch.float64, device=dev)
        O = None
        if with_O:
            O = torch.empty((B, self.nparams), dtype=torch.float64 if prec == "fp64" else torch.float32, device=dev)
        vjp = torch.empty(self.nparams, dtype=torch.float64, device=dev) if weights is not None else None
        w = weights.to(device=dev, dtype=torch.float64).contiguous() if weights is not None else None
        _check(_lib().dn_logpsi_grad(self._h, N, _ptr(spins), B, PRECISIONS[prec], _stream(stream), _ptr(lp),
                                     _ptr(O), _ptr(w), _ptr(vjp)), "dn_logpsi_grad")
        return lp, O, vjp

    def sampler_batch(self, spins: torch.Tensor, sites: torch.Tensor, u: torch.Tensor, eps: float, prec="fp32",
                      stream=None):
        """One batch of the screened typewriter sampler on C chains (spins [C][N] int8 updated in
        place; sites [C][K] int32 proposals, -1 = none; u [C][K] float64).  Returns
        (accepted [C][K] int8, {"proposals", "accepted", "refreshes"})."""
        C, N = spins.shape
        K = sites.shape[1]
        acc = torch.empty((C, K), dtype=torch.int8, device=spins.device)
        st = SamplerStats()
        _check(_lib().dn_sampler_batch(self._h, N, _ptr(spins), C, _ptr(sites), _ptr(u), K, float(eps),
                                       PRECISIONS[prec], _stream(stream), _ptr(acc), ctypes.byref(st)),
               "dn_sampler_batch")
        return acc, {"proposals": st.proposals, "accepted": st.accepted, "refreshes": st.refreshes}

    def recompute_flip_ratios(self, spins: torch.Tensor, sample: torch.Tensor, sites: torch.Tensor, prec="fp32",
                              stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
        B, N = spins.shape
        F = sample.shape[0]
        if out is None:
            out = torch.empty(F, dtype=torch.float64, device=spins.device)
        _check(_lib().dn_recompute_flip_ratios(self._h, N, _ptr(spins), B, _ptr(sample), _ptr(sites), F,
                                               PRECISIONS[prec], _stream(stream), _ptr(out)),
               "dn_recompute_flip_ratios")
        return out


class Cache:
    """Per-sample ABACUS caches built by dysonnet_forward_cache."""

    def __init__(self, model: Model, handle, spins):
        self.model, self._h = model, handle
        self.N, self.B = spins.shape[1], spins.shape[0]

    def flip_ratios(self, sample: torch.Tensor, sites: torch.Tensor, stream=None,
                    out: torch.Tensor | None = None) -> torch.Tensor:
        """abacus_flip_ratios: sample int32 [F], sites int32 [F][2] (-1 = unused)."""
        F = sample.shape[0]
        if out is None:
            out = torch.empty(F, dtype=torch.float64, device=sample.device)
        _check(_lib().abacus_flip_ratios(self._h, _ptr(sample), _ptr(sites), F, _ptr(out), _stream(stream)),
               "abacus_flip_ratios")
        return out

    def single_flip_ratios(self, stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
        """abacus_single_flip_ratios: [B][N] ratios of every single flip."""
        if out is None:
            out = torch.empty((self.B, self.N), dtype=torch.float64, device="cuda")
        _check(_lib().abacus_single_flip_ratios(self._h, _ptr(out), _stream(stream)), "abacus_single_flip_ratios")
        return out

    def pair_flip_ratios(self, bonds=(1, 2), stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
        """abacus_pair_flip_ratios: [B][len(bonds)][N] ratios of the pairs {j, j + bond}."""
        nb = len(bonds)
        arr = (ctypes.c_int32 * max(nb, 1))(*bonds)
        if out is None:
            out = torch.empty((self.B, nb, self.N), dtype=torch.float64, device="cuda")
        _check(_lib().abacus_pair_flip_ratios(self._h, nb, arr, _ptr(out), _stream(stream)),
               "abacus_pair_flip_ratios")
        return out

    def check(self, stream=None) -> int:
        return int(_lib().dn_cache_check(self._h, _stream(stream)))

    def tensor(self, name: str) -> torch.Tensor:
        """Copy of one cache array (inspection and debugging)."""
        ptr, cnt, eb = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_int()
        _check(_lib().dn_cache_tensor(self._h, name.encode(), ctypes.byref(ptr), ctypes.byref(cnt), ctypes.byref(eb)),
               "dn_cache_tensor")
        typestr = {1: "|i1", 4: "<f4", 8: "<f8"}[eb.value]
        if cnt.value == 0:
            return torch.empty(0, dtype={1: torch.int8, 4: torch.float32, 8: torch.float64}[eb.value], device="cuda")
        torch.cuda.current_stream().synchronize()
        return _device_view(ptr.value, cnt.value, typestr).clone()

    def destroy(self):
        if self._h is not None and self._h.value:
            _lib().dn_cache_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _device_view(ptr: int, count: int, typestr: str) -> torch.Tensor:
    """Non-owning torch view of library-owned device memory (callers copy it at once; torch
    accepts only views flagged writable)."""

    class _Arr:
        __cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (ptr, False), "version": 3}

    return torch.as_tensor(_Arr(), device="cuda")


class Server:
    """Continuous-batching request loop of the library (dn_server_*): chains of any N
    with resident caches, requests of single-site proposals served in batches by one
    kernel; mode "abacus", "persistent" (one resident kernel fed by a work queue) or
    "recompute" (full forward pass of every proposal)."""

    def __init__(self, model: "Model", prec="fp32", mode="abacus", hbm_budget_bytes: int = 16 << 30,
                 max_batch_flips: int = 8192, max_batch_chains: int = 64):
        self._model = model
        self._h = ctypes.c_void_p()
        m = {"abacus": DN_SERVE_ABACUS, "recompute": DN_SERVE_RECOMPUTE, "persistent": DN_SERVE_PERSISTENT}[mode]
        _check(_lib().dn_server_create(model._h, PRECISIONS[prec], m, int(hbm_budget_bytes), int(max_batch_flips),
                                       int(max_batch_chains), ctypes.byref(self._h)), "dn_server_create")
        self._out = {}

    def set_idle_limit(self, seconds: float):
        _check(_lib().dn_server_set_idle_limit(self._h, float(seconds)), "dn_server_set_idle_limit")

    def kernel_status(self, wait_s: float = 0.0):
        """(status, running) of the resident kernel of a persistent server."""
        run = ctypes.c_int()
        st = _lib().dn_server_kernel_status(self._h, float(wait_s), ctypes.byref(run))
        return st, bool(run.value)

    def set_chain(self, chain: int, spins, build_now: bool = False):
        import numpy as np
        a = np.ascontiguousarray(spins, dtype=np.int8)
        _check(_lib().dn_server_set_chain(self._h, int(chain), int(a.size), a.ctypes.data, int(bool(build_now))),
               "dn_server_set_chain")

    def submit(self, chain: int, sites) -> int:
        """sites: int array [F] of single sites or [F, 2] (second entry -1)."""
        import numpy as np
        x = np.asarray(sites, dtype=np.int32)
        if x.ndim == 1:
            x = np.stack([x, -np.ones_like(x)], axis=1)
        x = np.ascontiguousarray(x)
        out = np.empty(x.shape[0], dtype=np.float64)
        t = ctypes.c_ulonglong()
        _check(_lib().dn_server_submit(self._h, int(chain), x.ctypes.data, int(x.shape[0]), out.ctypes.data,
                                       ctypes.byref(t)), "dn_server_submit")
        self._out[t.value] = (out, x)
        return t.value

    def wait(self, ticket: int, timeout_s: float = -1.0):
        """(ratios, latency in seconds) of a submitted request."""
        lat = ctypes.c_double()
        st = _lib().dn_server_wait(self._h, ctypes.c_ulonglong(ticket), float(timeout_s), ctypes.byref(lat))
        if st == DN_ETIMEOUT:
            _check(st, "dn_server_wait")
        out, _ = self._out.pop(ticket)
        _check(st, "dn_server_wait")
        return out, lat.value

    def stats(self) -> dict:
        s = ServerStats()
        _check(_lib().dn_server_get_stats(self._h, ctypes.byref(s)), "dn_server_get_stats")
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            _lib().dn_server_destroy(self._h)
            self._h = ctypes.c_void_p()


def sr_matrices(O: torch.Tensor, gram: bool = True, block: tuple[int, int] | None = None, stream=None):
    """(Oc Oc^T / B or None, Oc[:, k0:k0+nk]^T Oc[:, k0:k0+nk] / B or None) for the log-derivatives
    O [B][nparams] (float64 or float32), Oc = O - mean over the samples."""
    B, P = O.shape
    prec = "fp64" if O.dtype == torch.float64 else "fp32"
    G = torch.empty((B, B), dtype=torch.float64, device=O.device) if gram else None
    S, k0, nk = None, 0, 0
    if block is not None:
        k0, nk = block
        S = torch.empty((nk, nk), dtype=torch.float64, device=O.device)
    _check(_lib().dn_sr_matrices(_ptr(O), B, P, PRECISIONS[prec], _stream(stream), _ptr(G), k0, nk, _ptr(S)),
           "dn_sr_matrices")
    return G, S


class LogPsi(torch.autograd.Function):
    """log psi(sigma_b) [B] as a differentiable function of the parameter vector theta
    (float64, the layout of dn_model_create).  The backward pass is the library's reverse
    pass: grad_theta = sum_b grad_out_b d log psi(sigma_b) / d theta (dn_logpsi_grad).

        lp = LogPsi.apply(theta, desc, spins, "fp64")
    """

    @staticmethod
    def forward(ctx, theta, desc, spins, prec="fp64"):
        model = Model(desc, theta.detach().cpu().numpy())
        lp = model.full_forward(spins, prec=prec)
        ctx.model, ctx.prec = model, prec
        ctx.save_for_backward(spins)
        ctx.theta_device = theta.device
        return lp.to(theta.device)

    @staticmethod
    def backward(ctx, grad_lp):
        (spins,) = ctx.saved_tensors
        _, _, vjp = ctx.model.logpsi_grad(spins, prec=ctx.prec, weights=grad_lp.to(spins.device), with_O=False)
        ctx.model.close()
        return vjp.to(ctx.theta_device), None, None, None
