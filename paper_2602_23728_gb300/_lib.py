"""ctypes binding of libphx.so: argument marshalling only.

Every computation happens inside the CUDA library.  Arrays may be NumPy arrays (host
memory) or CUDA torch tensors (device memory, enqueued on the current torch stream); all
array arguments of one call must live on the same side.  If the compiled library is
missing this module raises at import time: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libphx.so")

PHX_MEM_HOST, PHX_MEM_DEVICE = 0, 1
PHX_GAUSS, PHX_LORENTZ = 0, 1
PHX_FP64, PHX_TF32, PHX_BF16X3 = 0, 1, 2
STATUS = {0: "PHX_OK", 1: "PHX_ERR_INVALID", 2: "PHX_ERR_CUDA", 3: "PHX_ERR_NOMEM", 4: "PHX_ERR_TIMEOUT",
          5: "PHX_ERR_UNSUPPORTED", 6: "PHX_ERR_NUMERIC"}
PRECISIONS = {"fp64": PHX_FP64, "tf32": PHX_TF32, "bf16x3": PHX_BF16X3}
SHAPES = {"gauss": PHX_GAUSS, "lorentz": PHX_LORENTZ}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libphx.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python -m paper_2602_23728_gb300.build")
lib = C.CDLL(LIB_PATH)


class Cell(C.Structure):
    _fields_ = [("lattice", C.c_double * 9), ("n_atoms", C.c_int32), ("masses", C.c_void_p),
                ("positions", C.c_void_p)]


class Ifc2(C.Structure):
    _fields_ = [("n_blocks", C.c_int32), ("idx", C.c_void_p), ("val", C.c_void_p)]


class Ifc3(C.Structure):
    _fields_ = [("nnz", C.c_int64), ("idx", C.c_void_p), ("val", C.c_void_p)]


class Broadening(C.Structure):
    _fields_ = [("shape", C.c_int32), ("sigma_thz", C.c_double), ("window", C.c_double)]


class Job(C.Structure):
    _fields_ = [("fc3", C.c_void_p), ("freq_thz", C.c_void_p), ("evec", C.c_void_p), ("irr_q", C.c_void_p),
                ("n_irr", C.c_int32), ("temperature", C.c_double), ("br", Broadening), ("f_min_thz", C.c_double),
                ("gamma", C.c_void_p), ("irr_q_dev", C.c_void_p), ("full_to_irr", C.c_void_p), ("vv", C.c_void_p),
                ("gamma_full", C.c_void_p), ("volume", C.c_double), ("kappa", C.c_void_p)]


class Tune(C.Structure):
    _fields_ = [("q_tile", C.c_int32), ("chain", C.c_int32), ("side_sms", C.c_int32)]


_P = C.c_void_p
_I = C.c_int32
lib.phx_create.argtypes = [C.POINTER(_P), C.c_int]
lib.phx_create.restype = C.c_int
lib.phx_destroy.argtypes = [_P]
lib.phx_destroy.restype = None
lib.phx_last_error.argtypes = [_P]
lib.phx_last_error.restype = C.c_char_p
lib.phx_version.argtypes = []
lib.phx_version.restype = C.c_char_p
lib.phx_irreducible.argtypes = [_P, _I, _P, _P, _P, _P, _P]
lib.phx_irreducible.restype = C.c_int
lib.phx_harmonic.argtypes = [_P, C.POINTER(Cell), C.POINTER(Ifc2), _P, _I, _P, _P, _P, _P, _I, _P]
lib.phx_harmonic.restype = C.c_int
lib.phx_fc3_create.argtypes = [_P, C.POINTER(Cell), C.POINTER(Ifc3), _P, C.POINTER(_P)]
lib.phx_fc3_create.restype = C.c_int
lib.phx_fc3_destroy.argtypes = [_P]
lib.phx_fc3_destroy.restype = None
lib.phx_fc3_num_d.argtypes = [_P]
lib.phx_fc3_num_d.restype = C.c_int32
lib.phx_gamma.argtypes = [_P, _P, _P, _P, _P, _I, C.c_double, Broadening, C.c_double, _I, _P, _P, _I, _P]
lib.phx_gamma.restype = C.c_int
lib.phx_gamma_multi_t.argtypes = [_P, _P, _P, _P, _P, _I, _P, _I, Broadening, C.c_double, _I, _P, _I, _P]
lib.phx_gamma_multi_t.restype = C.c_int
lib.phx_gamma_isotope.argtypes = [_P, _I, _I, _P, _P, _P, _I, _P, Broadening, C.c_double, _P, _I, _P]
lib.phx_gamma_isotope.restype = C.c_int
lib.phx_kappa_qhgk.argtypes = [_P, C.POINTER(Cell), C.POINTER(Ifc2), _P, _P, _P, C.c_double, C.c_double, _P, _I, _P]
lib.phx_kappa_qhgk.restype = C.c_int
lib.phx_gamma_cell.argtypes = [_P, _P, _P, _P, C.c_double, Broadening, C.c_double, _I, _P, _I, _P]
lib.phx_gamma_cell.restype = C.c_int
lib.phx_unfold.argtypes = [_P, _I, _I, _I, _P, _P, _P, _P, _P, _I, _P]
lib.phx_unfold.restype = C.c_int
lib.phx_kappa_rta.argtypes = [_P, C.POINTER(Cell), _I, _I, _P, _P, _P, _P, C.c_double, C.c_double, _I, _P, _I, _P]
lib.phx_kappa_rta.restype = C.c_int
lib.phx_kappa_sc.argtypes = [_P, C.POINTER(Cell), _P, _P, _P, _P, C.c_double, Broadening, C.c_double, _I, _I,
                             C.c_double, _P, _P, _P, _P, _P, _P, _I, _P]
lib.phx_kappa_sc.restype = C.c_int

lib.phx_set_option.argtypes = [_P, _I, C.c_int64]
lib.phx_set_option.restype = C.c_int
lib.phx_get_option.argtypes = [_P, _I, C.c_void_p]
lib.phx_get_option.restype = C.c_int
lib.phx_profile_enable.argtypes = [_P, _I]
lib.phx_profile_enable.restype = C.c_int
lib.phx_profile_read.argtypes = [_P, _I, _P, _P, _P, _P]
lib.phx_profile_read.restype = C.c_int

lib.phx_kappa_rta_noalloc.argtypes = [C.POINTER(Cell), _I, _I, _P, _P, _P, _P, C.c_double, C.c_double, _I, _P, _P]
lib.phx_kappa_rta_noalloc.restype = C.c_int

lib.phx_gamma_batched.argtypes = [_P, _I, _P, _I, _P, _P]
lib.phx_gamma_batched.restype = C.c_int

lib.phx_features.argtypes = [_P, _P, _I, _P, _P, _P, _I, C.c_double, Broadening, C.c_double, _P, _P]
lib.phx_features.restype = C.c_int
lib.phx_mlp_create.argtypes = [_P, _I, _I, _I, _I, C.c_uint64, C.POINTER(_P)]
lib.phx_mlp_create.restype = C.c_int
lib.phx_mlp_destroy.argtypes = [_P]
lib.phx_mlp_destroy.restype = None
lib.phx_mlp_num_params.argtypes = [_P]
lib.phx_mlp_num_params.restype = C.c_int64
lib.phx_mlp_get_params.argtypes = [_P, _P, _P]
lib.phx_mlp_get_params.restype = C.c_int
lib.phx_mlp_set_params.argtypes = [_P, _P, _P]
lib.phx_mlp_set_params.restype = C.c_int
lib.phx_mlp_loss_grad.argtypes = [_P, _P, _P, _I, _P, _P, _P]
lib.phx_mlp_loss_grad.restype = C.c_int
lib.phx_mlp_train.argtypes = [_P, _P, _P, _I, _I, C.c_double, _P, _P]
lib.phx_mlp_train.restype = C.c_int
lib.phx_mlp_train_es.argtypes = [_P, _P, _P, _I, _I, _I, C.c_double, _I, _I, _P, _P, _P]
lib.phx_mlp_train_es.restype = C.c_int
lib.phx_mlp_predict.argtypes = [_P, _P, _I, _P, _P, _P]
lib.phx_mlp_predict.restype = C.c_int
lib.phx_mlp_reconstruct.argtypes = [_P, _I, _I, _P, _P, _P, _P, C.c_double, _P, _P, _P, _P]
lib.phx_mlp_outside.argtypes = [_P, _P, _I, _P, _P]
lib.phx_mlp_outside.restype = C.c_int
lib.phx_mlp_reconstruct.restype = C.c_int

KERNELS = {"dft": 0, "gemm_e2": 1, "gemm_e1_gamma": 2, "fold": 3, "fp64_gemm": 4, "fp64_epilogue": 5,
           "eigensolver": 6, "cell_sparse": 7, "cell_transpose": 8, "cell_gemm": 9, "eig_tridiag": 10,
           "eig_vectors": 11, "eig_back": 12, "eig_bisect": 13, "sc_step": 14, "chain": 15}

OPTIONS = {"chain": 0, "wait_limit_ns": 1, "starve": 2, "pair": 3, "side_sms": 4, "vel_fp32": 5, "harmonic_tr": 6, "sc_matrix_free": 7}

EXPORTED = ["phx_set_option", "phx_get_option", "phx_profile_enable", "phx_profile_read", "phx_create", "phx_destroy", "phx_last_error", "phx_version", "phx_irreducible", "phx_harmonic",
            "phx_fc3_create", "phx_fc3_destroy", "phx_fc3_num_d", "phx_gamma", "phx_gamma_multi_t", "phx_gamma_isotope", "phx_kappa_qhgk", "phx_gamma_cell", "phx_unfold", "phx_kappa_rta", "phx_kappa_sc",
            "phx_kappa_rta_noalloc", "phx_gamma_batched", "phx_features", "phx_mlp_create", "phx_mlp_destroy",
            "phx_mlp_num_params", "phx_mlp_get_params", "phx_mlp_set_params", "phx_mlp_loss_grad", "phx_mlp_train",
            "phx_mlp_predict", "phx_mlp_reconstruct", "phx_mlp_train_es", "phx_mlp_outside"]


class PhxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return x.data_ptr()
    return x.ctypes.data


def _host(x, dtype):
    a = np.ascontiguousarray(x, dtype=dtype)
    return a


def _mem_and_stream(arrays):
    dev = [a for a in arrays if a is not None and _is_torch(a)]
    if not dev:
        return PHX_MEM_HOST, None
    if len(dev) != len([a for a in arrays if a is not None]):
        raise ValueError("mix of host (numpy) and device (torch) arrays in one call")
    import torch
    for a in dev:
        if not a.is_cuda or not a.is_contiguous():
            raise ValueError("device arrays must be contiguous CUDA tensors")
    return PHX_MEM_DEVICE, torch.cuda.current_stream(dev[0].device).cuda_stream


def make_cell(lattice, masses):
    m = _host(masses, np.float64)
    c = Cell()
    for k, v in enumerate(np.asarray(lattice, dtype=np.float64).ravel()):
        c.lattice[k] = v
    c.n_atoms = m.shape[0]
    c.masses = m.ctypes.data
    c.positions = None
    return c, m


def time_reversal_count(mesh):
    """Number of orbits {q, -q} of a Gamma-centred mesh (the unknowns' q-points of
    phx_kappa_sc): the points with q = -q mod G (k_i in {0, n_i/2}) plus half of the rest."""
    n_self = int(np.prod([2 if int(k) % 2 == 0 else 1 for k in mesh]))
    return (int(np.prod([int(k) for k in mesh])) + n_self) // 2


def irreducible(mesh, rotations):
    """Irreducible set (host): returns irr, full_to_irr, weights as int32 arrays."""
    mesh_a = np.asarray(mesh, dtype=np.int32)
    rot = np.ascontiguousarray(rotations, dtype=np.int32).reshape(-1, 9)
    nq = int(np.prod(mesh_a))
    irr = np.zeros(nq, np.int32)
    f2i = np.zeros(nq, np.int32)
    wt = np.zeros(nq, np.int32)
    n_irr = C.c_int32(0)
    st = lib.phx_irreducible(mesh_a.ctypes.data, rot.shape[0], rot.ctypes.data, irr.ctypes.data,
                             C.addressof(n_irr), f2i.ctypes.data, wt.ctypes.data)
    if st != 0:
        raise PhxError(st, "phx_irreducible failed (rotation does not map the mesh onto itself?)")
    k = n_irr.value
    return irr[:k].copy(), f2i, wt[:k].copy()


class FC3:
    """Handle of prepared third-order IFCs (phx_fc3)."""

    def __init__(self, ctx, lattice, masses, idx, val, mesh):
        self.ctx = ctx
        self._idx = _host(idx, np.int32)
        self._val = _host(val, np.float64)
        cell, self._m = make_cell(lattice, masses)
        f = Ifc3(self._val.shape[0], self._idx.ctypes.data, self._val.ctypes.data)
        self._mesh = np.asarray(mesh, dtype=np.int32)
        h = _P()
        ctx._check(lib.phx_fc3_create(ctx.h, C.byref(cell), C.byref(f), self._mesh.ctypes.data, C.byref(h)))
        self.h = h
        self.n = 3 * self._m.shape[0]
        self.mesh = tuple(int(x) for x in mesh)
        self.nq = int(np.prod(self._mesh))

    @property
    def num_d(self):
        return lib.phx_fc3_num_d(self.h)

    def close(self):
        if self.h:
            lib.phx_fc3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One phx context on a CUDA device."""

    def __init__(self, device=0):
        h = _P()
        st = lib.phx_create(C.byref(h), int(device))
        if st != 0:
            raise PhxError(st, "phx_create failed (no CUDA device?)")
        self.h = h
        self.device = device

    def _check(self, st):
        if st != 0:
            raise PhxError(st, lib.phx_last_error(self.h).decode())

    def close(self):
        if self.h:
            lib.phx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ profiling
    def set_option(self, name, value):
        """Context option: 'chain' (0 auto, 1 chained kernel wherever it fits, 2 never),
        'pair' (1: one evaluation per exchange pair {q', q''}, 0: every q'),
        'side_sms' (SMs of the fold/Fourier side stream next to the contractions; -1 default, 0 off),
        'vel_fp32' (1: velocity products of harmonic() with FP32 products and sums),
        'harmonic_tr' (1, default: harmonic() solves one q of each {q, -q} pair and fills the other
        by time reversal; 0: every q solved on its own),
        'sc_matrix_free' (kappa_sc's Gamma1: 0 dense when it fits, else matrix-free; 1 always
        matrix-free; 2 always dense),
        'wait_limit_ns' (bound of every device barrier wait), 'starve' (test hook)."""
        self._check(lib.phx_set_option(self.h, OPTIONS[name], int(value)))

    def get_option(self, name):
        """The option's value in effect ('side_sms': the SM count the tensor-core path gives its side stream)."""
        v = C.c_int64(0)
        self._check(lib.phx_get_option(self.h, OPTIONS[name], C.addressof(v)))
        return int(v.value)

    def profile_enable(self, on=True):
        self._check(lib.phx_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """{kernel: (total_ms, launches, flops, bytes)} plus 'launches' (all kernels)."""
        out = {}
        for name, k in KERNELS.items():
            ms, n, fl, by = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
            self._check(lib.phx_profile_read(self.h, k, C.addressof(ms), C.addressof(n), C.addressof(fl),
                                             C.addressof(by)))
            out[name] = (ms.value, n.value, fl.value, by.value)
        n = C.c_int64()
        self._check(lib.phx_profile_read(self.h, -1, None, C.addressof(n), None, None))
        out["launches"] = n.value
        return out

    # ------------------------------------------------------------------ harmonic
    def harmonic(self, lattice, masses, ifc2_idx, ifc2_val, q_frac, freq=None, evec=None, vel=None, vv=None,
                 want_vel=True, want_vv=True):
        """phx_harmonic.  With numpy q_frac, outputs are allocated as numpy arrays; with a CUDA
        tensor q_frac the caller passes CUDA tensors for the outputs."""
        cell, m = make_cell(lattice, masses)
        bi = _host(ifc2_idx, np.int32)
        bv = _host(ifc2_val, np.float64)
        f2 = Ifc2(bi.shape[0], bi.ctypes.data, bv.ctypes.data)
        n = 3 * m.shape[0]
        if not _is_torch(q_frac):
            q_frac = _host(q_frac, np.float64).reshape(-1, 3)
            nq = q_frac.shape[0]
            freq = np.zeros((nq, n)) if freq is None else freq
            evec = np.zeros((nq, n, n), np.complex128) if evec is None else evec
            if want_vel and vel is None:
                vel = np.zeros((nq, n, 3))
            if want_vv and vv is None:
                vv = np.zeros((nq, n, 3, 3))
        nq = q_frac.shape[0]
        mem, stream = _mem_and_stream([q_frac, freq, evec, vel, vv])
        self._check(lib.phx_harmonic(self.h, C.byref(cell), C.byref(f2), _ptr(q_frac), nq, _ptr(freq), _ptr(evec),
                                     _ptr(vel), _ptr(vv), mem, stream))
        return freq, evec, vel, vv

    # ------------------------------------------------------------------ scattering
    def fc3(self, lattice, masses, idx, val, mesh):
        return FC3(self, lattice, masses, idx, val, mesh)

    def gamma(self, fc3, freq, evec, irr_q, temperature, shape="gauss", sigma=0.1, window=2.0, f_min=0.01,
              precision="fp64", gamma=None, wp2=None, want_wp2=False):
        br = Broadening(SHAPES[shape], float(sigma), float(window))
        if not _is_torch(freq):
            freq = _host(freq, np.float64)
            evec = _host(evec, np.complex128)
            irr_q = _host(irr_q, np.int32)
            gamma = np.zeros((irr_q.shape[0], fc3.n)) if gamma is None else gamma
            if want_wp2 and wp2 is None:
                wp2 = np.zeros((irr_q.shape[0], fc3.n))
        mem, stream = _mem_and_stream([freq, evec, irr_q, gamma, wp2])
        self._check(lib.phx_gamma(self.h, fc3.h, _ptr(freq), _ptr(evec), _ptr(irr_q), int(irr_q.shape[0]),
                                  float(temperature), br, float(f_min), PRECISIONS[precision], _ptr(gamma),
                                  _ptr(wp2), mem, stream))
        return (gamma, wp2) if want_wp2 or wp2 is not None else gamma

    def gamma_multi_t(self, fc3, freq, evec, irr_q, temperatures, shape="gauss", sigma=0.1, window=2.0, f_min=0.01,
                      precision="bf16x3", gamma=None):
        """phx_gamma_multi_t: gamma[n_t][n_irr][n] for several temperatures from one contraction."""
        br = Broadening(SHAPES[shape], float(sigma), float(window))
        temps = _host(temperatures, np.float64).reshape(-1)
        if not _is_torch(freq):
            freq = _host(freq, np.float64)
            evec = _host(evec, np.complex128)
            irr_q = _host(irr_q, np.int32)
            gamma = np.zeros((temps.shape[0], irr_q.shape[0], fc3.n)) if gamma is None else gamma
        mem, stream = _mem_and_stream([freq, evec, irr_q, gamma])
        self._check(lib.phx_gamma_multi_t(self.h, fc3.h, _ptr(freq), _ptr(evec), _ptr(irr_q), int(irr_q.shape[0]),
                                          temps.ctypes.data, int(temps.shape[0]), br, float(f_min),
                                          PRECISIONS[precision], _ptr(gamma), mem, stream))
        return gamma

    def gamma_isotope(self, freq, evec, irr_q, g_atom, shape="gauss", sigma=0.1, window=2.0, f_min=0.01,
                      gamma=None):
        """phx_gamma_isotope: Tamura mass-variance rates [n_irr][n] (freq [nq, n], evec [nq, n, n])."""
        br = Broadening(SHAPES[shape], float(sigma), float(window))
        g = _host(g_atom, np.float64).reshape(-1)
        nq, n = int(freq.shape[0]), int(freq.shape[1])
        if not _is_torch(freq):
            freq = _host(freq, np.float64)
            evec = _host(evec, np.complex128)
            irr_q = _host(irr_q, np.int32)
            gamma = np.zeros((irr_q.shape[0], n)) if gamma is None else gamma
        mem, stream = _mem_and_stream([freq, evec, irr_q, gamma])
        self._check(lib.phx_gamma_isotope(self.h, nq, n, _ptr(freq), _ptr(evec), _ptr(irr_q), int(irr_q.shape[0]),
                                          g.ctypes.data, br, float(f_min), _ptr(gamma), mem, stream))
        return gamma

    def gamma_cell(self, fc3, freq, evec, temperature, shape="lorentz", sigma=0.1, window=2.0, f_min=0.01,
                   precision="bf16x3", gamma=None):
        """phx_gamma_cell: Gamma-only linewidths of every mode of a large cell (fc3 made for a
        1x1x1 mesh; freq [n], evec [n, n] complex with zero imaginary parts)."""
        br = Broadening(SHAPES[shape], float(sigma), float(window))
        if not _is_torch(freq):
            freq = _host(freq, np.float64).reshape(-1)
            evec = _host(evec, np.complex128)
            gamma = np.zeros(fc3.n) if gamma is None else gamma
        mem, stream = _mem_and_stream([freq, evec, gamma])
        self._check(lib.phx_gamma_cell(self.h, fc3.h, _ptr(freq), _ptr(evec), float(temperature), br, float(f_min),
                                       PRECISIONS[precision], _ptr(gamma), mem, stream))
        return gamma

    def gamma_batched(self, jobs, precision="bf16x3", q_tiles=None, chain=None, side_sms=None):
        """phx_gamma_batched.  jobs: list of dicts with keys fc3 (FC3), freq, evec (CUDA tensors),
        irr (numpy int32), irr_dev (CUDA int32), T, shape, sigma, window, f_min, gamma (CUDA out),
        and optionally vv, full_to_irr, gamma_full, kappa (CUDA) and volume for the conductivity.
        q_tiles: None (autotune the tile, the contraction kernel and the side-stream share) or a
        list of q' tiles per job; chain, side_sms: with q_tiles, lists per job (chain: 1 chained
        kernel, 0 two GEMMs; side_sms: SMs of the side stream, 0 one stream; -1 the context
        option) or None (-1 for all).  Returns the (q_tile, chain, side_sms) used per job."""
        import torch
        arr = (Job * len(jobs))()
        keep = []
        for k, j in enumerate(jobs):
            irr = _host(j["irr"], np.int32)
            keep.append(irr)
            a = arr[k]
            a.fc3 = j["fc3"].h
            a.freq_thz = _ptr(j["freq"])
            a.evec = _ptr(j["evec"])
            a.irr_q = irr.ctypes.data
            a.n_irr = irr.shape[0]
            a.temperature = float(j["T"])
            a.br = Broadening(SHAPES[j.get("shape", "gauss")], float(j.get("sigma", 0.1)), float(j.get("window", 2.0)))
            a.f_min_thz = float(j.get("f_min", 0.01))
            a.gamma = _ptr(j["gamma"])
            a.irr_q_dev = _ptr(j["irr_dev"])
            a.full_to_irr = _ptr(j.get("full_to_irr"))
            a.vv = _ptr(j.get("vv"))
            a.gamma_full = _ptr(j.get("gamma_full"))
            a.volume = float(j.get("volume", 0.0))
            a.kappa = _ptr(j.get("kappa"))
        tune = (Tune * max(1, len(jobs)))()
        for k in range(len(jobs)):
            tune[k].q_tile = 0 if q_tiles is None else int(q_tiles[k])
            tune[k].chain = -1 if chain is None else int(chain[k])
            tune[k].side_sms = -1 if side_sms is None else int(side_sms[k])
        dev = jobs[0]["freq"].device if jobs else torch.device("cuda", self.device)
        stream = torch.cuda.current_stream(dev).cuda_stream
        self._check(lib.phx_gamma_batched(self.h, len(jobs), C.addressof(arr), PRECISIONS[precision],
                                          C.addressof(tune), stream))
        return [(tune[k].q_tile, tune[k].chain, tune[k].side_sms) for k in range(len(jobs))]

    # ------------------------------------------------------------------ learned linewidths
    def features(self, mesh, freq, vel, irr_dev, temperature, shape="gauss", sigma=0.1, window=2.0, f_min=0.01,
                 out=None):
        """phx_features on CUDA tensors: out [n_irr][n][4] (created when None)."""
        import torch
        mesh_a = np.asarray(mesh, dtype=np.int32)
        n = freq.shape[1]
        if out is None:
            out = torch.zeros((irr_dev.shape[0], n, 4), dtype=torch.float64, device=freq.device)
        br = Broadening(SHAPES[shape], float(sigma), float(window))
        stream = torch.cuda.current_stream(freq.device).cuda_stream
        self._check(lib.phx_features(self.h, mesh_a.ctypes.data, n, _ptr(freq), _ptr(vel), _ptr(irr_dev),
                                     int(irr_dev.shape[0]), float(temperature), br, float(f_min), _ptr(out), stream))
        return out

    def mlp(self, n_in=4, width=128, depth=3, ensemble=4, seed=0):
        return MLP(self, n_in, width, depth, ensemble, seed)

    def mlp_reconstruct(self, n, mean, std, wp2, freq_rows, f_min=0.01, outside=None):
        """phx_mlp_reconstruct on CUDA tensors: (gamma [rows], score [rows / n]) from the
        ensemble's log prediction (wp2 None: no residual factor; outside: int32 flags from
        MLP.outside, which make their q-point's score infinite)."""
        import torch
        rows = mean.shape[0]
        if rows % n:
            raise ValueError("mlp_reconstruct: rows must be a multiple of n")
        for a in (mean, std, wp2, freq_rows):
            if a is not None and (not a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous()
                                  or a.numel() != rows):
                raise ValueError("mlp_reconstruct: contiguous float64 CUDA tensors of one row count")
        if outside is not None and (not outside.is_cuda or outside.dtype != torch.int32 or not outside.is_contiguous()
                                    or outside.numel() != rows):
            raise ValueError("mlp_reconstruct: outside must be a contiguous int32 CUDA tensor of the row count")
        gamma = torch.empty(rows, dtype=torch.float64, device=mean.device)
        score = torch.empty(rows // n, dtype=torch.float64, device=mean.device) if std is not None else None
        self._check(lib.phx_mlp_reconstruct(self.h, rows // n, n, _ptr(mean), _ptr(std), _ptr(wp2), _ptr(freq_rows),
                                            float(f_min), _ptr(outside), _ptr(gamma), _ptr(score),
                                            torch.cuda.current_stream(mean.device).cuda_stream))
        return gamma, score

    # ------------------------------------------------------------------ transport
    def unfold(self, freq_full, irr_q, gamma_irr, full_to_irr, out=None):
        """phx_unfold: irreducible linewidths (degenerate-averaged) onto the full mesh."""
        if not _is_torch(freq_full):
            freq_full = _host(freq_full, np.float64)
            irr_q = _host(irr_q, np.int32)
            gamma_irr = _host(gamma_irr, np.float64)
            full_to_irr = _host(full_to_irr, np.int32)
            out = np.zeros((full_to_irr.shape[0], freq_full.shape[1])) if out is None else out
        mem, stream = _mem_and_stream([freq_full, irr_q, gamma_irr, full_to_irr, out])
        self._check(lib.phx_unfold(self.h, gamma_irr.shape[0], full_to_irr.shape[0], freq_full.shape[1],
                                   _ptr(freq_full), _ptr(irr_q), _ptr(gamma_irr), _ptr(full_to_irr), _ptr(out),
                                   mem, stream))
        return out

    def kappa_qhgk(self, lattice, masses, positions, ifc2_idx, ifc2_val, freq, evec, gamma, temperature,
                   f_min=0.01):
        """phx_kappa_qhgk: Gamma-only QHGK conductivity (3 x 3, W/(m K)) of a cell; freq [n],
        evec [n, n] complex with zero imaginary parts, gamma [n] (numpy or CUDA tensors)."""
        cell, m = make_cell(lattice, masses)
        pos = _host(positions, np.float64).reshape(-1, 3)
        cell.positions = pos.ctypes.data
        bi = _host(ifc2_idx, np.int32)
        bv = _host(ifc2_val, np.float64)
        f2 = Ifc2(bi.shape[0], bi.ctypes.data, bv.ctypes.data)
        if not _is_torch(freq):
            freq = _host(freq, np.float64).reshape(-1)
            evec = _host(evec, np.complex128)
            gamma = _host(gamma, np.float64).reshape(-1)
        mem, stream = _mem_and_stream([freq, evec, gamma])
        k = np.zeros(9)
        self._check(lib.phx_kappa_qhgk(self.h, C.byref(cell), C.byref(f2), _ptr(freq), _ptr(evec), _ptr(gamma),
                                       float(temperature), float(f_min), k.ctypes.data, mem, stream))
        return k.reshape(3, 3)

    def kappa_rta(self, lattice, masses, freq, gamma_full, temperature, vel=None, vv=None, f_min=0.01,
                  is_classic=False):
        cell, m = make_cell(lattice, masses)
        if not _is_torch(freq):
            freq = _host(freq, np.float64)
            gamma_full = _host(gamma_full, np.float64)
            vel = None if vel is None else _host(vel, np.float64)
            vv = None if vv is None else _host(vv, np.float64)
        mem, stream = _mem_and_stream([freq, gamma_full, vel, vv])
        k = np.zeros(9)
        self._check(lib.phx_kappa_rta(self.h, C.byref(cell), freq.shape[0], freq.shape[1], _ptr(freq), _ptr(vel),
                                      _ptr(vv), _ptr(gamma_full), float(temperature), float(f_min), int(is_classic),
                                      k.ctypes.data, mem, stream))
        return k.reshape(3, 3)


    def kappa_sc(self, lattice, masses, fc3, freq, evec, vel, temperature, shape="gauss", sigma=0.1, window=2.0,
                 f_min=0.01, precision="bf16x3", max_iter=100, tol=1e-6, want_gamma1=False, gamma0=None, mfp=None,
                 gamma1=None):
        """phx_kappa_sc: the iterative BTE on the time-reversal representatives of fc3's mesh.
        Returns dict(kappa [k+1, 3, 3] (iterate 0 = RTA), n_iter, converged, gamma0 [n_tr, n],
        mfp [n_tr, n, 3], gamma1 [R, R] or None)."""
        br = Broadening(SHAPES[shape], float(sigma), float(window))
        cell, m = make_cell(lattice, masses)
        n_tr = time_reversal_count(fc3.mesh)
        R = n_tr * fc3.n
        if not _is_torch(freq):
            freq = _host(freq, np.float64)
            evec = _host(evec, np.complex128)
            vel = _host(vel, np.float64)
            gamma0 = np.zeros((n_tr, fc3.n)) if gamma0 is None else gamma0
            mfp = np.zeros((n_tr, fc3.n, 3)) if mfp is None else mfp
            if want_gamma1 and gamma1 is None:
                gamma1 = np.zeros((R, R))
        mem, stream = _mem_and_stream([freq, evec, vel, gamma0, mfp, gamma1])
        hist = np.zeros((int(max_iter) + 1) * 9)
        n_it = C.c_int32(0)
        conv = C.c_int32(0)
        self._check(lib.phx_kappa_sc(self.h, C.byref(cell), fc3.h, _ptr(freq), _ptr(evec), _ptr(vel),
                                     float(temperature), br, float(f_min), PRECISIONS[precision], int(max_iter),
                                     float(tol), hist.ctypes.data, C.addressof(n_it), C.addressof(conv),
                                     _ptr(gamma0), _ptr(mfp), _ptr(gamma1), mem, stream))
        k = n_it.value
        return dict(kappa=hist[:9 * (k + 1)].reshape(k + 1, 3, 3), n_iter=k, converged=bool(conv.value),
                    gamma0=gamma0, mfp=mfp, gamma1=gamma1)


class MLP:
    """Handle of a phx_mlp ensemble (device parameters; device inputs)."""

    def __init__(self, ctx, n_in, width, depth, ensemble, seed):
        h = _P()
        ctx._check(lib.phx_mlp_create(ctx.h, n_in, width, depth, ensemble, int(seed), C.byref(h)))
        self.ctx, self.h = ctx, h
        self.n_in, self.width, self.depth, self.ensemble = n_in, width, depth, ensemble
        self.n_params = int(lib.phx_mlp_num_params(h))

    def _stream(self, x):
        import torch
        return torch.cuda.current_stream(x.device).cuda_stream

    def get_params(self):
        p = np.zeros((self.ensemble, self.n_params), np.float32)
        nrm = np.zeros(2 * self.n_in + 2, np.float32)
        self.ctx._check(lib.phx_mlp_get_params(self.h, p.ctypes.data, nrm.ctypes.data))
        return p, nrm

    def set_params(self, params, norm=None):
        p = np.ascontiguousarray(params, np.float32)
        nrm = None if norm is None else np.ascontiguousarray(norm, np.float32)
        self.ctx._check(lib.phx_mlp_set_params(self.h, p.ctypes.data, None if nrm is None else nrm.ctypes.data))

    def loss_grad(self, X, y):
        loss = np.zeros(self.ensemble)
        g = np.zeros((self.ensemble, self.n_params), np.float32)
        self.ctx._check(lib.phx_mlp_loss_grad(self.h, _ptr(X), _ptr(y), int(X.shape[0]), loss.ctypes.data,
                                              g.ctypes.data, self._stream(X)))
        return loss, g

    def train(self, X, y, epochs, lr=3e-3):
        loss = np.zeros(self.ensemble)
        self.ctx._check(lib.phx_mlp_train(self.h, _ptr(X), _ptr(y), int(X.shape[0]), int(epochs), float(lr),
                                          loss.ctypes.data, self._stream(X)))
        return loss

    def train_es(self, X, y, n_val, max_epochs, lr=3e-3, check_every=50, patience=4):
        """Early-stopped training: the last n_val rows of X, y are the held-out set.  Returns
        (final training loss per member, epochs run)."""
        loss = np.zeros(self.ensemble)
        ran = C.c_int32(0)
        self.ctx._check(lib.phx_mlp_train_es(self.h, _ptr(X), _ptr(y), int(X.shape[0]), int(n_val), int(max_epochs),
                                             float(lr), int(check_every), int(patience), loss.ctypes.data,
                                             C.addressof(ran), self._stream(X)))
        return loss, ran.value

    def predict(self, X, mean=None, std=None):
        import torch
        rows = X.shape[0]
        mean = torch.zeros(rows, dtype=torch.float64, device=X.device) if mean is None else mean
        std = torch.zeros(rows, dtype=torch.float64, device=X.device) if std is None else std
        self.ctx._check(lib.phx_mlp_predict(self.h, _ptr(X), rows, _ptr(mean), _ptr(std), self._stream(X)))
        return mean, std

    def outside(self, X, out=None):
        """int32 flag per row of X (CUDA float64 [rows][n_in]): 1 where an input lies outside the
        range of the last training rows."""
        import torch
        if not X.is_cuda or X.dtype != torch.float64 or not X.is_contiguous() or X.dim() != 2 or X.shape[1] != self.n_in:
            raise ValueError("outside: X must be a contiguous float64 CUDA tensor [rows][n_in]")
        rows = X.shape[0]
        out = torch.zeros(rows, dtype=torch.int32, device=X.device) if out is None else out
        self.ctx._check(lib.phx_mlp_outside(self.h, _ptr(X), rows, _ptr(out), self._stream(X)))
        return out

    def close(self):
        if self.h:
            lib.phx_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kappa_rta_noalloc(lattice, masses, freq, gamma_full, temperature, out, vel=None, vv=None, f_min=0.01,
                      is_classic=False):
    """phx_kappa_rta_noalloc: device tensors in, kappa into the device tensor `out` (9 doubles);
    enqueued on the current torch stream, no device allocation inside the library."""
    cell, m = make_cell(lattice, masses)
    arrays = [freq, gamma_full, vel, vv, out]
    if not all(a is None or (_is_torch(a) and a.is_cuda and a.is_contiguous()) for a in arrays):
        raise ValueError("phx_kappa_rta_noalloc takes contiguous CUDA tensors only")
    import torch
    if any(a is not None and a.dtype != torch.float64 for a in arrays):
        raise ValueError("phx_kappa_rta_noalloc takes float64 tensors only")
    if any(a is not None and a.device != freq.device for a in arrays):
        raise ValueError("phx_kappa_rta_noalloc: all tensors must be on one device")
    if freq.dim() != 2 or tuple(gamma_full.shape) != tuple(freq.shape):
        raise ValueError("phx_kappa_rta_noalloc: freq and gamma_full must both be [nq, n]")
    if (vel is None) == (vv is None):
        raise ValueError("phx_kappa_rta_noalloc: give exactly one of vel [nq, n, 3] and vv [nq, n, 3, 3]")
    if vel is not None and tuple(vel.shape) != tuple(freq.shape) + (3,):
        raise ValueError("phx_kappa_rta_noalloc: vel must be [nq, n, 3]")
    if vv is not None and tuple(vv.shape) != tuple(freq.shape) + (3, 3):
        raise ValueError("phx_kappa_rta_noalloc: vv must be [nq, n, 3, 3]")
    if out.numel() < 9:
        raise ValueError("phx_kappa_rta_noalloc: out must hold 9 doubles")
    # the library takes its scratch array's address on the current device: make it the tensors'
    with torch.cuda.device(freq.device):
        stream = torch.cuda.current_stream(freq.device).cuda_stream
        st = lib.phx_kappa_rta_noalloc(C.byref(cell), freq.shape[0], freq.shape[1], _ptr(freq), _ptr(vel), _ptr(vv),
                                       _ptr(gamma_full), float(temperature), float(f_min), int(is_classic),
                                       _ptr(out), stream)
    if st != 0:
        raise PhxError(st, "phx_kappa_rta_noalloc failed")
    return out


def version():
    return lib.phx_version().decode()
