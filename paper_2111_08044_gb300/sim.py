"""User-facing wrapper: a chain state in a torch CUDA tensor driven through
the C ABI.  Torch provides device memory and the stream; every step of the
evolution runs in libfloquetsv's kernels."""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import numpy as np

from . import capi


class FloquetSimulator:
    """One open chain of L sites on one GPU.

    >>> sim = FloquetSimulator(L=12)
    >>> sim.init_product_state(spinors)          # (L, 4) float64
    >>> sim.build(J=1.0, hx=0.9, hz=0.4, T=0.5, K=4, theta=0.3)
    >>> e, n = sim.evolve(100)                   # energy density, norm per period
    """

    def __init__(self, L: int, precision: str = "c64", device: int = 0, stream=None,
                 state=None):
        import torch
        self._torch = torch
        self.L = int(L)
        # df64: double-float check mode; its buffer holds (hi, lo) FP32 pairs
        # in complex128-sized elements, read out as complex128 by state_c128()
        precisions = {"c64": capi.SV_C64, "c128": capi.SV_C128, "df64": capi.SV_DF64}
        if precision not in precisions:
            raise ValueError(f"precision must be one of {sorted(precisions)}")
        self.precision = precisions[precision]
        dtype = torch.complex64 if self.precision == capi.SV_C64 else torch.complex128
        self.device = torch.device("cuda", device)
        if state is None:
            state = torch.empty(1 << self.L, dtype=dtype, device=self.device)
        if state.dtype != dtype or not state.is_cuda or not state.is_contiguous():
            raise ValueError("state must be a contiguous CUDA tensor of the matching dtype")
        self.state = state
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._lib = capi.load()
        ctx = ctypes.c_void_p()
        capi.check(self._lib.sv_create(ctypes.byref(ctx), self.device.index or 0,
                                       self.precision, ctypes.c_void_p(self.stream.cuda_stream)),
                   None, "sv_create")
        self._ctx = ctx
        capi.check(self._lib.sv_attach_state(ctx, ctypes.c_void_p(state.data_ptr()),
                                             state.numel() * state.element_size()),
                   ctx, "sv_attach_state")
        self._keep = []

    # -- lifecycle
    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.sv_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def init_product_state(self, spinors: np.ndarray):
        sp = np.ascontiguousarray(spinors, dtype=np.float64)
        if sp.shape != (self.L, 4):
            raise ValueError(f"spinors must be ({self.L}, 4)")
        capi.check(self._lib.sv_init(self._ctx, self.L, sp.ctypes.data_as(capi._dp)),
                   self._ctx, "sv_init")

    def build(self, **kw):
        p, keep = capi.make_params(**kw)
        self._keep = keep
        capi.check(self._lib.sv_build_floquet(self._ctx, ctypes.byref(p)), self._ctx,
                   "sv_build_floquet")

    def evolve(self, periods: int, record: bool = True) -> Tuple[np.ndarray, np.ndarray]:
        e = np.zeros(max(periods, 1))
        n = np.zeros(max(periods, 1))
        ep = e.ctypes.data_as(capi._dp) if record else None
        np_ = n.ctypes.data_as(capi._dp) if record else None
        capi.check(self._lib.sv_evolve(self._ctx, int(periods), ep, np_), self._ctx,
                   "sv_evolve")
        return e[:periods], n[:periods]

    def keep_period_layout(self, keep: bool = True):
        """Between evolve calls keep the state in the block plan's period
        layout (sv_set_layout_policy): saves one relabel pass per call; the
        calls that read the state restore the natural layout first."""
        capi.check(self._lib.sv_set_layout_policy(self._ctx, 1 if keep else 0), self._ctx,
                   "sv_set_layout_policy")

    def save(self, path: str):
        """Checkpoint the state and the period counter (sv_save)."""
        capi.check(self._lib.sv_save(self._ctx, str(path).encode()), self._ctx, "sv_save")

    def load(self, path: str):
        """Resume from a checkpoint (sv_load): state, L and period counter."""
        capi.check(self._lib.sv_load(self._ctx, str(path).encode()), self._ctx, "sv_load")

    def energy(self) -> Tuple[float, float]:
        e = ctypes.c_double()
        n = ctypes.c_double()
        capi.check(self._lib.sv_expect_energy(self._ctx, ctypes.byref(e), ctypes.byref(n)),
                   self._ctx, "sv_expect_energy")
        return e.value, n.value

    def energy_moments(self) -> Tuple[float, float, float]:
        """(E, sigma_E, |psi|^2) of the current state: E = <H0> and sigma_E =
        sqrt(<H0^2> - E^2) on the normalised state (Eq. 10, Eq. 11)."""
        e, s, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        capi.check(self._lib.sv_energy_moments(self._ctx, ctypes.byref(e), ctypes.byref(s),
                                               ctypes.byref(n)), self._ctx, "sv_energy_moments")
        return e.value, s.value, n.value

    def overlap_product(self, spinors: np.ndarray) -> complex:
        """<phi|psi> with the product state phi of `spinors` ((L, 4) as for
        init_product_state; each site normalised)."""
        sp = np.ascontiguousarray(spinors, dtype=np.float64)
        re, im = ctypes.c_double(), ctypes.c_double()
        capi.check(self._lib.sv_overlap_product(self._ctx, sp.ctypes.data_as(capi._dp),
                                                ctypes.byref(re), ctypes.byref(im)),
                   self._ctx, "sv_overlap_product")
        return complex(re.value, im.value)

    def init_pairs(self, pair_states: np.ndarray):
        """Dimer-product initial state over the site pairs (2k, 2k+1):
        pair_states is (L/2, 4) complex, local index r = 2 b_2k + b_2k+1."""
        ps = np.ascontiguousarray(pair_states, dtype=np.complex128)
        assert ps.shape == (self.L // 2, 4)
        capi.check(self._lib.sv_init_pairs(self._ctx, self.L, ps.ctypes.data_as(capi._dp)),
                   self._ctx, "sv_init_pairs")

    def overlap_pairs(self, pair_states: np.ndarray) -> complex:
        """<phi|psi> with the dimer-product state of pair_states."""
        ps = np.ascontiguousarray(pair_states, dtype=np.complex128)
        re, im = ctypes.c_double(), ctypes.c_double()
        capi.check(self._lib.sv_overlap_pairs(self._ctx, ps.ctypes.data_as(capi._dp),
                                              ctypes.byref(re), ctypes.byref(im)),
                   self._ctx, "sv_overlap_pairs")
        return complex(re.value, im.value)

    def renormalize(self) -> float:
        n = ctypes.c_double()
        capi.check(self._lib.sv_renormalize(self._ctx, ctypes.byref(n)), self._ctx,
                   "sv_renormalize")
        return n.value

    def adjoint(self, periods: Optional[int] = None) -> Tuple[np.ndarray, np.ndarray, float]:
        """Gradients of the energy density after `periods` periods (default:
        all per-period parameters) with respect to those periods' kick angles
        and fields, and that energy density."""
        P = self._n_period_params() if periods is None else int(periods)
        gt = np.zeros(max(P, 0))
        gh = np.zeros(max(P, 0))
        e = ctypes.c_double()
        capi.check(self._lib.sv_adjoint(self._ctx, P, gt.ctypes.data_as(capi._dp),
                                        gh.ctypes.data_as(capi._dp), ctypes.byref(e)),
                   self._ctx, "sv_adjoint")
        return gt, gh, e.value

    def _n_period_params(self) -> int:
        sizes = [k.size for k in self._keep]
        return max(sizes) if sizes else 0

    def state_c128(self):
        """The state as a complex128 CUDA tensor: the buffer itself (c128) or
        a copy converted by the library (df64, c64)."""
        torch = self._torch
        if self.precision == capi.SV_C128:
            return self.state
        if self.precision == capi.SV_C64:
            return self.state.to(torch.complex128)
        out = torch.empty(1 << self.L, dtype=torch.complex128, device=self.device)
        capi.check(self._lib.sv_get_state(self._ctx, ctypes.c_void_p(out.data_ptr()),
                                          out.numel() * out.element_size()),
                   self._ctx, "sv_get_state")
        return out

    def host_state(self) -> np.ndarray:
        dt = np.complex64 if self.precision == capi.SV_C64 else np.complex128
        out = np.empty(1 << self.L, dtype=dt)
        capi.check(self._lib.sv_get_state(self._ctx, ctypes.c_void_p(out.ctypes.data),
                                          out.nbytes), self._ctx, "sv_get_state")
        return out

    def set_host_state(self, psi: np.ndarray, period: int = 0):
        dt = np.complex64 if self.precision == capi.SV_C64 else np.complex128
        a = np.ascontiguousarray(psi, dtype=dt)
        capi.check(self._lib.sv_set_state(self._ctx, ctypes.c_void_p(a.ctypes.data), a.nbytes,
                                          int(period)), self._ctx, "sv_set_state")

    @property
    def period(self) -> int:
        return int(self._lib.sv_period_counter(self._ctx))

    def evolve_profiled(self, periods: int):
        """(energy, norm, per-launch milliseconds summed over the periods)."""
        p, _, nl = self.pass_info()
        e = np.zeros(max(periods, 1))
        n = np.zeros(max(periods, 1))
        ms = np.zeros(nl)
        capi.check(self._lib.sv_evolve_profiled(self._ctx, int(periods), e.ctypes.data_as(capi._dp),
                                                n.ctypes.data_as(capi._dp),
                                                ms.ctypes.data_as(capi._dp)),
                   self._ctx, "sv_evolve_profiled")
        return e[:periods], n[:periods], ms

    def form_info(self):
        """(tensor_cores, block_n) of the built evolution."""
        tc, n = ctypes.c_int(), ctypes.c_int()
        capi.check(self._lib.sv_form_info(self._ctx, ctypes.byref(tc), ctypes.byref(n)),
                   self._ctx, "sv_form_info")
        return bool(tc.value), n.value

    def build_bytes(self) -> int:
        b = ctypes.c_size_t()
        capi.check(self._lib.sv_build_bytes(self._ctx, ctypes.byref(b)), self._ctx,
                   "sv_build_bytes")
        return b.value

    def pass_info(self):
        p, g, l = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        capi.check(self._lib.sv_pass_info(self._ctx, ctypes.byref(p), ctypes.byref(g),
                                          ctypes.byref(l)), self._ctx, "sv_pass_info")
        return p.value, g.value, l.value


def chain_params(cfg, **over):
    """Keyword arguments of FloquetSimulator.build for a ChainConfig."""
    kw = dict(J=cfg.J, hx=cfg.hx, hz=cfg.hz, T=cfg.T, theta=cfg.theta,
              edge_field_weight=cfg.edge_field_weight, K=cfg.K, first_layer=cfg.first_layer)
    if getattr(cfg, "theta_p", None) is not None:
        kw["theta_p"] = cfg.theta_p
    if getattr(cfg, "hx_p", None) is not None:
        kw["hx_p"] = cfg.hx_p
    kw.update(over)
    return kw


class FloquetBatch:
    """Many independent chains (uneven L, per-chain parameters) evolved
    together on one GPU through the batch calls of the C ABI.

    >>> b = FloquetBatch(inputs.batch_preset(512))
    >>> e, n = b.evolve(100)          # [n_chains, periods] each
    >>> b.forms()                     # SV_BATCH_* form per chain
    """

    def __init__(self, chains, form: int = capi.SV_BATCH_AUTO, device: int = 0, stream=None):
        import torch
        self._torch = torch
        self.n = len(chains)
        self.L = np.array([c.L for c in chains], dtype=np.int32)
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._lib = capi.load()
        total = int(self._lib.sv_batch_state_bytes(self.n, self.L.ctypes.data_as(capi._ip)))
        if total == 0:
            raise ValueError("chain sizes must be in 2..34")
        self.state = torch.empty(total, dtype=torch.uint8, device=self.device)
        params = (capi.sv_floquet_params * self.n)()
        for k, c in enumerate(chains):
            p, _ = capi.make_params(J=c.J, hx=c.hx, hz=c.hz, T=c.T, theta=c.theta,
                                    edge_field_weight=c.edge_field_weight, K=c.K,
                                    first_layer=c.first_layer)
            params[k] = p
        self._params = params
        sp = np.ascontiguousarray(np.concatenate([c.spinors().reshape(-1) for c in chains]),
                                  dtype=np.float64)
        b = ctypes.c_void_p()
        rc = self._lib.sv_batch_create(ctypes.byref(b), self.device.index or 0, self.n,
                                       self.L.ctypes.data_as(capi._ip), params,
                                       sp.ctypes.data_as(capi._dp),
                                       ctypes.c_void_p(self.state.data_ptr()), total, int(form),
                                       ctypes.c_void_p(self.stream.cuda_stream))
        if rc != capi.SV_OK:
            raise capi.SvError(rc, "sv_batch_create")
        self._b = b
        self.offsets = []
        off = 0
        for L in self.L:
            off = (off + 255) // 256 * 256
            self.offsets.append(off)
            off += 8 << int(L)

    def close(self):
        if getattr(self, "_b", None):
            self._lib.sv_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc, what):
        if rc != capi.SV_OK:
            m = self._lib.sv_batch_last_error(self._b)
            raise capi.SvError(rc, f"{what}: {m.decode() if m else ''}")

    def evolve(self, periods: int):
        e = np.zeros((self.n, max(periods, 1)))
        nn = np.zeros((self.n, max(periods, 1)))
        self._check(self._lib.sv_batch_evolve(self._b, int(periods), e.ctypes.data_as(capi._dp),
                                              nn.ctypes.data_as(capi._dp)), "sv_batch_evolve")
        return e[:, :periods], nn[:, :periods]

    def forms(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int32)
        self._check(self._lib.sv_batch_forms(self._b, out.ctypes.data_as(capi._ip)),
                    "sv_batch_forms")
        return out

    def widths(self) -> np.ndarray:
        """Block width n of each chain's form (0 for non-block forms)."""
        out = np.zeros(self.n, dtype=np.int32)
        self._check(self._lib.sv_batch_widths(self._b, out.ctypes.data_as(capi._ip)),
                    "sv_batch_widths")
        return out

    def chain_state(self, c: int) -> np.ndarray:
        """Host copy of chain c's complex64 state."""
        self._torch.cuda.synchronize(self.device)
        L = int(self.L[c])
        raw = self.state[self.offsets[c]:self.offsets[c] + (8 << L)]
        return raw.view(self._torch.complex64).cpu().numpy()
