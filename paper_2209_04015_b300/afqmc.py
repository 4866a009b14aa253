"""ctypes binding of libafqmc (include/afqmc.h): argument marshalling only.

Every entry point keeps the C name without its ``afq_`` prefix.  Host arrays are
numpy arrays (complex arrays as complex128, which matches the interleaved
(re, im) doubles of the C ABI); the ``*_dev`` methods take raw device pointers
(for example ``tensor.data_ptr()``).  There is no fallback: if the library
cannot be loaded, ``load_library`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libafqmc.so")

AFQ_OK, AFQ_ERR_ARG, AFQ_ERR_CUDA, AFQ_ERR_SINGULAR, AFQ_ERR_NAN, AFQ_ERR_STATE, AFQ_ERR_NOMEM = range(7)
AFQ_STATIC_EXCHANGE_SLOTS = 262144  # complex partial-sum slots of the static scratch array
PRECISIONS = {"fp64": 0, "split_bf16": 1, "split_tf32": 2}
EXCHANGES = {"auto": 0, "direct": 1, "stored": 2}
PROP_KERNELS = {"per_pass": 0, "fused": 1, "per_pair": 2}
STATUS_NAMES = {0: "AFQ_OK", 1: "AFQ_ERR_ARG", 2: "AFQ_ERR_CUDA", 3: "AFQ_ERR_SINGULAR",
                4: "AFQ_ERR_NAN", 5: "AFQ_ERR_STATE", 6: "AFQ_ERR_NOMEM"}


class AfqParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("taylor_order", ctypes.c_int),
                ("qr_period", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int), ("has_e_shift", ctypes.c_int),
                ("e_shift", ctypes.c_double), ("fb_cap", ctypes.c_double),
                ("free_projection", ctypes.c_int), ("split_slices", ctypes.c_int),
                ("prop_slices", ctypes.c_int), ("exchange", ctypes.c_int),
                ("prop_kernel", ctypes.c_int)]


class AfqError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "afq_default_params": (None, [ctypes.POINTER(AfqParams)]),
    "afq_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(AfqParams), _P]),
    "afq_destroy": (ctypes.c_int, [_P]),
    "afq_last_error": (ctypes.c_char_p, [_P]),
    "afq_init_hamiltonian": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_double]),
    "afq_init_trial": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "afq_trial_energy": (ctypes.c_int, [_P, _D]),
    "afq_exchange_algorithm": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "afq_prop_digits": (ctypes.c_int, [_P, _P, ctypes.c_int, _D]),
    "afq_init_walkers": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "afq_propagate": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "afq_propagate_dev": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "afq_local_energy": (ctypes.c_int, [_P, _P, _D]),
    "afq_local_energy_dev": (ctypes.c_int, [_P, _P, _P]),
    "afq_orthogonalise": (ctypes.c_int, [_P]),
    "afq_comb": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _P]),
    "afq_run_blocks": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_double,
                                      ctypes.c_int, _P]),
    "afq_get_e_shift": (ctypes.c_int, [_P, _P]),
    "afq_spin_squared": (ctypes.c_int, [_P, _P, _P]),
    "afq_one_rdm": (ctypes.c_int, [_P, _P]),
    "afq_local_energy_backward": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "afq_local_energy_backward_dev": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "afq_chain_forward": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "afq_chain_forward_dev": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "afq_chain_backward": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "afq_chain_backward_dev": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "afq_get_walkers": (ctypes.c_int, [_P, _P]),
    "afq_get_weights": (ctypes.c_int, [_P, _P]),
    "afq_get_overlaps": (ctypes.c_int, [_P, _P]),
    "afq_get_force_bias": (ctypes.c_int, [_P, _P]),
    "afq_get_step": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "afq_set_state": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_uint64]),
    "afq_philox_fields": (ctypes.c_int, [_P, ctypes.c_uint64, _P]),
    "afq_philox_words": (ctypes.c_int, [_P, ctypes.c_uint64, _P]),
    "afq_launch_count": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "afq_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "afq_profile_read": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_uint64)]),
    "afq_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
    "afq_graph_capture": (ctypes.c_int, [_P, ctypes.c_int]),
    "afq_graph_launch": (ctypes.c_int, [_P, ctypes.c_int]),
    "afq_get_energy": (ctypes.c_int, [_P, _P, _D]),
    "afq_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)]),
    "afq_batch_destroy": (ctypes.c_int, [_P]),
    "afq_batch_last_error": (ctypes.c_char_p, [_P]),
    "afq_batch_capture": (ctypes.c_int, [_P, ctypes.c_int]),
    "afq_batch_set_grouped": (ctypes.c_int, [_P, ctypes.c_int]),
    "afq_batch_launch": (ctypes.c_int, [_P, ctypes.c_int]),
    "afq_batch_synchronize": (ctypes.c_int, [_P]),
    "afq_autotune": (ctypes.c_int, [_P]),
    "afq_get_tiles": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "afq_gemm_split_bf16": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            _P, _P, _P, _P]),
    "afq_fp64_fma_rate": (ctypes.c_int, [_D, _P]),
    "afq_exchange_energy_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libafqmc.so and declare its signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libafqmc.so not built ({path}); run "
                           "`python -m paper_2209_04015_b300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exchange_energy_static(M: int, X: int, na: int, nb: int, W: int, Lt_ptr: int,
                           thetaT_ptr: int, ek_ptr: int, stream: int | None = None) -> None:
    """afq_exchange_energy_static on device pointers: exchange energy per walker with
    no device allocation (partial sums in the library's static scratch array)."""
    lib = load_library()
    rc = lib.afq_exchange_energy_static(M, X, na, nb, W, _P(Lt_ptr), _P(thetaT_ptr), _P(ek_ptr),
                                        _P(stream or 0))
    if rc != AFQ_OK:
        raise AfqError(rc, "afq_exchange_energy_static failed (details on stderr)")


def fp64_fma_rate(stream_ptr: int | None = None) -> float:
    """afq_fp64_fma_rate: measured FP64 FMA throughput of the current device, TFLOP/s."""
    lib = load_library()
    out = ctypes.c_double()
    rc = lib.afq_fp64_fma_rate(ctypes.byref(out), _P(stream_ptr) if stream_ptr else None)
    if rc != AFQ_OK:
        raise AfqError(rc, "afq_fp64_fma_rate failed")
    return out.value


def gemm_split_bf16(m: int, n: int, k: int, slices: int, A_ptr: int, B_ptr: int, C_ptr: int,
                    stream: int | None = None) -> None:
    """afq_gemm_split_bf16 on device pointers: C = A B^T in split-bf16 on the tensor cores."""
    lib = load_library()
    rc = lib.afq_gemm_split_bf16(m, n, k, slices, _P(A_ptr), _P(B_ptr), _P(C_ptr), _P(stream or 0))
    if rc != AFQ_OK:
        raise AfqError(rc, "afq_gemm_split_bf16 failed")


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_P)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


class AfqContext:
    """One walker ensemble on the current CUDA device (wraps afq_ctx*)."""

    def __init__(self, dt: float = 0.005, taylor_order: int = 6, qr_period: int = 5,
                 seed: int = 1, precision: str = "fp64", e_shift: float | None = None,
                 fb_cap: float = 0.0, free_projection: bool = False, stream: int | None = None,
                 split_slices: int = 4, prop_slices: int = 4, exchange: str = "auto",
                 prop_kernel: str = "per_pass"):
        self.lib = load_library()
        p = AfqParams()
        self.lib.afq_default_params(ctypes.byref(p))
        p.dt, p.taylor_order, p.qr_period, p.seed = dt, taylor_order, qr_period, seed
        p.precision = PRECISIONS[precision]
        p.has_e_shift = 0 if e_shift is None else 1
        p.e_shift = 0.0 if e_shift is None else float(e_shift)
        p.fb_cap = fb_cap
        p.free_projection = 1 if free_projection else 0
        p.split_slices = split_slices
        p.prop_slices = prop_slices
        p.exchange = EXCHANGES[exchange]
        p.prop_kernel = PROP_KERNELS[prop_kernel]
        self.params = p
        h = _P()
        rc = self.lib.afq_create(ctypes.byref(h), ctypes.byref(p), _P(stream or 0))
        if rc != AFQ_OK:
            raise AfqError(rc, "afq_create failed")
        self.h = h
        self.stream = stream or 0
        self.M = self.X = self.na = self.nb = self.W = 0

    # -- plumbing ---------------------------------------------------------------
    def _check(self, rc: int) -> None:
        if rc != AFQ_OK:
            raise AfqError(rc, self.lib.afq_last_error(self.h).decode())

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.afq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def N(self) -> int:
        return self.na + self.nb

    # -- entry points -------------------------------------------------------------
    def init_hamiltonian(self, h1: np.ndarray, L: np.ndarray, e0: float = 0.0) -> None:
        h1 = _c(h1, np.float64)
        L = _c(L, np.float64)
        self.M, self.X = h1.shape[0], L.shape[0]
        self._check(self.lib.afq_init_hamiltonian(self.h, self.M, self.X, _ptr(h1), _ptr(L),
                                                  float(e0)))

    def init_trial(self, psi_a: np.ndarray, psi_b: np.ndarray) -> None:
        a = _c(psi_a, np.float64)
        b = _c(psi_b, np.float64)
        self.na, self.nb = a.shape[1], b.shape[1]
        self._check(self.lib.afq_init_trial(self.h, self.na, self.nb, _ptr(a), _ptr(b)))

    def trial_energy(self) -> float:
        e = ctypes.c_double()
        self._check(self.lib.afq_trial_energy(self.h, ctypes.byref(e)))
        return e.value

    def exchange_algorithm(self) -> str:
        """The exchange algorithm the trial resolved to: "direct" or "stored"."""
        a = ctypes.c_int()
        self._check(self.lib.afq_exchange_algorithm(self.h, ctypes.byref(a)))
        return {v: k for k, v in EXCHANGES.items()}[a.value]

    def prop_digits(self) -> tuple[list[int], float]:
        """Split precision: exact digits per propagation pass (first P, the Taylor
        powers, last P) and the sqrt(dt) |V|_2 estimate they were chosen for."""
        n = self.params.taylor_order + 2
        d = (ctypes.c_int * n)()
        x = ctypes.c_double()
        self._check(self.lib.afq_prop_digits(self.h, ctypes.cast(d, _P), n, ctypes.byref(x)))
        return list(d), x.value

    def init_walkers(self, W: int, phi: np.ndarray | None = None,
                     w: np.ndarray | None = None) -> None:
        ph = None if phi is None else _c(phi, np.complex128)
        ww = None if w is None else _c(w, np.float64)
        self.W = W
        self._check(self.lib.afq_init_walkers(self.h, W, _ptr(ph), _ptr(ww)))

    def propagate(self, fields: np.ndarray | None = None, nsteps: int = 1) -> None:
        f = None if fields is None else _c(fields, np.float64)
        if f is not None and f.size != nsteps * self.W * self.X:
            raise ValueError("fields must hold nsteps x W x X values")
        self._check(self.lib.afq_propagate(self.h, _ptr(f), nsteps))

    def propagate_dev(self, fields_ptr: int | None, nsteps: int = 1) -> None:
        self._check(self.lib.afq_propagate_dev(self.h, _P(fields_ptr or 0) if fields_ptr else None,
                                               nsteps))

    def local_energy(self) -> tuple[np.ndarray, float]:
        e = np.empty((self.W, 4), dtype=np.complex128)
        emix = ctypes.c_double()
        self._check(self.lib.afq_local_energy(self.h, _ptr(e), ctypes.byref(emix)))
        return e, emix.value

    def local_energy_dev(self, e_ptr: int | None, emix_ptr: int | None) -> None:
        self._check(self.lib.afq_local_energy_dev(self.h, _P(e_ptr) if e_ptr else None,
                                                  _P(emix_ptr) if emix_ptr else None))

    def orthogonalise(self) -> None:
        self._check(self.lib.afq_orthogonalise(self.h))

    def comb(self, u: float, w_cap: float = 0.0) -> np.ndarray:
        """Population control by the comb with offset u in [0, 1); returns the parent
        index of every new walker."""
        parents = np.empty(self.W, dtype=np.int32)
        self._check(self.lib.afq_comb(self.h, float(u), float(w_cap), _ptr(parents)))
        return parents

    def run_blocks(self, nblocks: int, steps_per_block: int = 25,
                   u: np.ndarray | None = None, w_cap: float = 0.0,
                   shift_feedback: bool = False) -> np.ndarray:
        """Blocks of steps_per_block steps, each followed by the local energy, the energy
        shift feedback (when asked) and, when u is given (one offset per block), the
        comb.  Returns (nblocks, 4): Re, Im of sum w and Re, Im of sum w E_L per block."""
        sums = np.empty((nblocks, 4), dtype=np.float64)
        uu = None if u is None else _c(u, np.float64)
        if uu is not None and uu.size != nblocks:
            raise ValueError("one comb offset per block")
        self._check(self.lib.afq_run_blocks(self.h, int(nblocks), int(steps_per_block),
                                            _ptr(uu), float(w_cap), 1 if shift_feedback else 0,
                                            _ptr(sums)))
        return sums

    def spin_squared(self) -> tuple[np.ndarray, float]:
        """Mixed <S^2> per walker (complex) and the weighted estimate."""
        out = np.empty(self.W, dtype=np.complex128)
        mix = ctypes.c_double()
        self._check(self.lib.afq_spin_squared(self.h, _ptr(out), ctypes.byref(mix)))
        return out, mix.value

    def one_rdm(self) -> np.ndarray:
        """Weighted mixed one-body density matrix, (2, M, M) complex (alpha, beta)."""
        out = np.empty((2, self.M, self.M), dtype=np.complex128)
        self._check(self.lib.afq_one_rdm(self.h, _ptr(out)))
        return out

    def get_e_shift(self) -> float:
        """The energy shift of the weight update (E_HF of the trial unless set or fed
        back by run_blocks)."""
        out = ctypes.c_double()
        self._check(self.lib.afq_get_e_shift(self.h, ctypes.byref(out)))
        return out.value

    def local_energy_backward(self, gE: np.ndarray, want=("h1", "L", "phi")):
        """Gradients of sum_z Re(conj(gE_z) E_L,z) at the current walkers: (dh1 (M, M),
        dL (X, M, M), dphi (W, M, N) complex), None for outputs not in ``want``."""
        g = _c(gE, np.complex128)
        if g.size != self.W:
            raise ValueError("gE must hold W complex values")
        dh = np.empty((self.M, self.M)) if "h1" in want else None
        dL = np.empty((self.X, self.M, self.M)) if "L" in want else None
        dp = np.empty((self.W, self.M, self.N), dtype=np.complex128) if "phi" in want else None
        self._check(self.lib.afq_local_energy_backward(self.h, _ptr(g), _ptr(dh), _ptr(dL),
                                                       _ptr(dp)))
        return dh, dL, dp

    def chain_forward(self, K: int, fields: np.ndarray | None = None) -> np.ndarray:
        """K steps with a tape for chain_backward; returns the energies (W, 4) at the end."""
        f = None if fields is None else _c(fields, np.float64)
        if f is not None and f.size != K * self.W * self.X:
            raise ValueError("fields must hold K x W x X values")
        e = np.empty((self.W, 4), dtype=np.complex128)
        self._check(self.lib.afq_chain_forward(self.h, K, _ptr(f), _ptr(e)))
        return e

    def chain_forward_dev(self, K: int, fields_ptr: int | None, e_ptr: int | None) -> None:
        self._check(self.lib.afq_chain_forward_dev(self.h, K, _P(fields_ptr) if fields_ptr else None,
                                                   _P(e_ptr) if e_ptr else None))

    def chain_backward(self, gE: np.ndarray, want=("h1", "L", "phi")):
        """Gradients of sum_z Re(conj(gE_z) E_L(Phi_z^K)) for the chain on the tape:
        (dh1 (M, M), dL (X, M, M)) symmetrised and dphi0 (W, M, N) complex."""
        g = _c(gE, np.complex128)
        if g.size != self.W:
            raise ValueError("gE must hold W complex values")
        dh = np.empty((self.M, self.M)) if "h1" in want else None
        dL = np.empty((self.X, self.M, self.M)) if "L" in want else None
        dp = np.empty((self.W, self.M, self.N), dtype=np.complex128) if "phi" in want else None
        self._check(self.lib.afq_chain_backward(self.h, _ptr(g), _ptr(dh), _ptr(dL), _ptr(dp)))
        return dh, dL, dp

    def chain_backward_dev(self, gE_ptr: int, dh1_ptr: int | None, dL_ptr: int | None,
                           dphi0_ptr: int | None) -> None:
        self._check(self.lib.afq_chain_backward_dev(
            self.h, _P(gE_ptr), _P(dh1_ptr) if dh1_ptr else None, _P(dL_ptr) if dL_ptr else None,
            _P(dphi0_ptr) if dphi0_ptr else None))

    def local_energy_backward_dev(self, gE_ptr: int, dh1_ptr: int | None, dL_ptr: int | None,
                                  dphi_ptr: int | None) -> None:
        self._check(self.lib.afq_local_energy_backward_dev(
            self.h, _P(gE_ptr), _P(dh1_ptr) if dh1_ptr else None, _P(dL_ptr) if dL_ptr else None,
            _P(dphi_ptr) if dphi_ptr else None))

    def get_walkers(self) -> np.ndarray:
        out = np.empty((self.W, self.M, self.N), dtype=np.complex128)
        self._check(self.lib.afq_get_walkers(self.h, _ptr(out)))
        return out

    def get_weights(self) -> np.ndarray:
        out = np.empty(self.W, dtype=np.complex128)
        self._check(self.lib.afq_get_weights(self.h, _ptr(out)))
        return out

    def get_overlaps(self) -> np.ndarray:
        out = np.empty(self.W, dtype=np.complex128)
        self._check(self.lib.afq_get_overlaps(self.h, _ptr(out)))
        return out

    def get_force_bias(self) -> np.ndarray:
        out = np.empty((self.W, self.X), dtype=np.complex128)
        self._check(self.lib.afq_get_force_bias(self.h, _ptr(out)))
        return out

    def get_step(self) -> int:
        s = ctypes.c_uint64()
        self._check(self.lib.afq_get_step(self.h, ctypes.byref(s)))
        return s.value

    def set_state(self, phi: np.ndarray, w: np.ndarray, ovlp: np.ndarray | None = None,
                  step: int = 0) -> None:
        ph = _c(phi, np.complex128)
        ww = _c(w, np.complex128)
        ov = None if ovlp is None else _c(ovlp, np.complex128)
        self._check(self.lib.afq_set_state(self.h, _ptr(ph), _ptr(ww), _ptr(ov), step))

    def philox_fields(self, step: int) -> np.ndarray:
        out = np.empty((self.W, self.X), dtype=np.float64)
        self._check(self.lib.afq_philox_fields(self.h, step, _ptr(out)))
        return out

    def philox_words(self, step: int) -> np.ndarray:
        out = np.empty((self.W, (self.X + 1) // 2, 4), dtype=np.uint32)
        self._check(self.lib.afq_philox_words(self.h, step, _ptr(out)))
        return out

    def profile_enable(self, on: bool = True) -> None:
        self._check(self.lib.afq_profile_enable(self.h, 1 if on else 0))

    def profile_read(self) -> dict[str, tuple[float, int]]:
        """{kernel class: (total ms, launches)} since profile_enable(True)."""
        out = {}
        k = 0
        while True:
            name = self.lib.afq_kernel_name(k)
            if name is None:
                break
            ms = ctypes.c_double()
            n = ctypes.c_uint64()
            self._check(self.lib.afq_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n)))
            out[name.decode()] = (ms.value, n.value)
            k += 1
        return out

    def graph_capture(self, nsteps: int) -> None:
        """Capture nsteps Philox steps + local energies as one CUDA graph."""
        self._check(self.lib.afq_graph_capture(self.h, nsteps))

    def graph_launch(self, nreplays: int = 1) -> None:
        self._check(self.lib.afq_graph_launch(self.h, nreplays))

    def get_energy(self) -> tuple[np.ndarray, float]:
        """Energies of the last evaluation (e.g. the last graph replay)."""
        e = np.empty((self.W, 4), dtype=np.complex128)
        emix = ctypes.c_double()
        self._check(self.lib.afq_get_energy(self.h, _ptr(e), ctypes.byref(emix)))
        return e, emix.value

    def autotune(self) -> None:
        self._check(self.lib.afq_autotune(self.h))

    def get_tiles(self) -> list[int]:
        """FP64 exchange g-group, FP64 propagator columns, split exchange walkers per
        tile (alpha, beta), force-bias split-K depth."""
        t = (ctypes.c_int * 5)()
        self._check(self.lib.afq_get_tiles(self.h, t, 5))
        return list(t)

    def launch_count(self) -> int:
        c = ctypes.c_uint64()
        self._check(self.lib.afq_launch_count(self.h, ctypes.byref(c)))
        return c.value


class AfqBatch:
    """Several contexts stepped by one CUDA graph (wraps afq_batch*): one concurrent
    branch per system, or with grouped=True (FP64 contexts) one persistent launch
    each for the VHS build and the propagation of all systems per step.  The
    contexts must outlive the batch."""

    def __init__(self, contexts: list[AfqContext], grouped: bool = False):
        self.lib = load_library()
        self.contexts = list(contexts)
        arr = (_P * len(self.contexts))(*[c.h for c in self.contexts])
        h = _P()
        rc = self.lib.afq_batch_create(ctypes.byref(h), len(self.contexts), arr)
        if rc != AFQ_OK:
            raise AfqError(rc, "afq_batch_create failed")
        self.h = h
        if grouped:
            self.set_grouped(True)

    def set_grouped(self, grouped: bool) -> None:
        """Launch layout of the next capture: per-system branches, or (FP64 contexts)
        grouped VHS and propagation launches over all systems."""
        self._check(self.lib.afq_batch_set_grouped(self.h, int(bool(grouped))))

    def _check(self, rc: int) -> None:
        if rc != AFQ_OK:
            raise AfqError(rc, self.lib.afq_batch_last_error(self.h).decode())

    def capture(self, nsteps: int) -> None:
        self._check(self.lib.afq_batch_capture(self.h, nsteps))

    def launch(self, nreplays: int = 1) -> None:
        self._check(self.lib.afq_batch_launch(self.h, nreplays))

    def synchronize(self) -> None:
        self._check(self.lib.afq_batch_synchronize(self.h))

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.afq_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
