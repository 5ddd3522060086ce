"""ctypes binding of libttn (include/ttn.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts NumPy
arrays to pointers and status codes to exceptions.  There is no fallback: if
the shared library is missing, importing it raises.
"""
import ctypes
import os

import numpy as np

from .workloads import PULSE_DTYPE

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libttn.so")

STATUS = {0: "TTN_OK", 1: "TTN_ERR_ARG", 2: "TTN_ERR_ALLOC", 3: "TTN_ERR_CUDA", 4: "TTN_ERR_KRYLOV",
          5: "TTN_ERR_NUMERIC", 6: "TTN_ERR_TIMEOUT", 7: "TTN_ERR_STATE"}
FP64, SPLIT_TF32X3 = 0, 1

# (name, restype, argtypes) for every symbol declared in include/ttn.h
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_I64 = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = [
    ("ttn_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)]),
    ("ttn_destroy", None, [_P]),
    ("ttn_last_error", ctypes.c_char_p, [_P]),
    ("ttn_set_stream", ctypes.c_int, [_P, _P]),
    ("ttn_set_precision", ctypes.c_int, [_P, ctypes.c_int]),
    ("ttn_set_hamiltonian", ctypes.c_int, [_P, _D, ctypes.c_double, ctypes.c_double]),
    ("ttn_apply_pulse", ctypes.c_int, [_P, _P, ctypes.c_int]),
    ("ttn_set_decay", ctypes.c_int, [_P, ctypes.c_double]),
    ("ttn_compress", ctypes.c_int, [_P, _P, _D]),
    ("ttn_sample", ctypes.c_int, [_P, _D, ctypes.c_int, _I]),
    ("ttn_fidelity_gradient", ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _I, _I,
                                              ctypes.c_int, ctypes.c_int, _D, _D]),
    ("ttn_set_product_state", ctypes.c_int, [_P, _D]),
    ("ttn_set_ghz_target", ctypes.c_int, [_P, _I, ctypes.c_double]),
    ("ttn_tdvp_step", ctypes.c_int, [_P, ctypes.c_double]),
    ("ttn_fidelity", ctypes.c_int, [_P, _P, _D]),
    ("ttn_overlap", ctypes.c_int, [_P, _P, _D]),
    ("ttn_measure", ctypes.c_int, [_P, ctypes.c_int, _D]),
    ("ttn_norm", ctypes.c_int, [_P, _D]),
    ("ttn_energy", ctypes.c_int, [_P, _D]),
    ("ttn_get_time", ctypes.c_int, [_P, _D]),
    ("ttn_get_dense", ctypes.c_int, [_P, _D]),
    ("ttn_save", ctypes.c_int, [_P, ctypes.c_char_p]),
    ("ttn_load", ctypes.c_int, [_P, ctypes.c_char_p]),
    ("ttn_num_nodes", ctypes.c_int, [_P, _I]),
    ("ttn_node_info", ctypes.c_int, [_P, ctypes.c_int, _I, _I]),
    ("ttn_leaf_atoms", ctypes.c_int, [_P, _I, _I]),
    ("ttn_get_node", ctypes.c_int, [_P, ctypes.c_int, _D]),
    ("ttn_set_node", ctypes.c_int, [_P, ctypes.c_int, _D]),
    ("ttn_refresh_envs", ctypes.c_int, [_P]),
    ("ttn_apply_heff", ctypes.c_int, [_P, ctypes.c_int, _D, _D]),
    ("ttn_get_stats", ctypes.c_int, [_P, _I64]),
    ("ttn_profile_begin", ctypes.c_int, [_P]),
    ("ttn_selftest_contract", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_ulonglong, ctypes.c_int, _D]),
    ("ttn_profile_end", ctypes.c_int, [_P, _D, ctypes.c_int]),
    ("ttn_selftest_qr", ctypes.c_int, [_D, ctypes.c_int, ctypes.c_int, _I, ctypes.c_int, _D, _D, _I,
                                       ctypes.POINTER(ctypes.c_float)]),
    ("ttn_profile_records", ctypes.c_int, [_P, _D, ctypes.c_int, _I]),
    ("ttn_reset_stats", ctypes.c_int, [_P]),
    ("ttn_contract_split_noalloc", ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    ("ttn_selftest_contract_host", ctypes.c_int, [_D, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, _I, ctypes.POINTER(ctypes.c_float)]),
    ("ttn_selftest_fp64_peak", ctypes.c_int, [ctypes.c_int, _D]),
    ("ttn_test_inject", ctypes.c_int, [ctypes.c_int, ctypes.c_longlong]),
    ("ttn_svd_truncate", ctypes.c_int, [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D, _D,
                                        _I, _D]),
]

# fault-injection hooks of ttn_test_inject
INJECT_NONE, INJECT_TC_STALL, INJECT_KRYLOV_MMAX, INJECT_ALLOC_FAIL = 0, 1, 2, 3

_lib = None


def load(path=LIB_PATH):
    """Load libttn.so (build it first with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libttn.so not found at %s: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def selftest_contract(M, N, K, precision, seed=1, tf32_exact=False):
    """max|C_p - C_fp64| / max|C_fp64| for one random M x K x N contraction."""
    lib = load()
    out = np.zeros(1)
    st = lib.ttn_selftest_contract(M, N, K, int(precision), seed, int(tf32_exact), _dptr(out))
    if st != 0:
        raise TTNError(st, "selftest_contract")
    return float(out[0])


def selftest_qr(A, cand=None):
    """GPU QR with deterministic completion of a host complex M x D matrix:
    returns (Q, R, n_dependent, device ms)."""
    lib = load()
    A = np.asfortranarray(np.asarray(A, dtype=np.complex128))
    M, D = A.shape
    Q = np.zeros((M, D), dtype=np.complex128, order="F")
    R = np.zeros((D, D), dtype=np.complex128, order="F")
    nd = ctypes.c_int(0)
    ms = ctypes.c_float(0.0)
    if cand is None:
        cp, nc = None, 0
    else:
        ca = np.ascontiguousarray(cand, dtype=np.int32)
        cp, nc = ca.ctypes.data_as(_I), len(ca)
    st = lib.ttn_selftest_qr(A.ctypes.data_as(_D), M, D, cp, nc, Q.ctypes.data_as(_D), R.ctypes.data_as(_D),
                             ctypes.byref(nd), ctypes.byref(ms))
    if st != 0:
        raise TTNError(st, "selftest_qr(%d, %d)" % (M, D))
    return Q, R, nd.value, ms.value


def contract_host(A, B, precision):
    """C = A B of host complex matrices on the device (FP64 kernel, or the
    split-precision tensor-core path when the shape fills its tiles): returns
    (C, tensor_core_path_ran, device ms)."""
    lib = load()
    A = np.asfortranarray(np.asarray(A, dtype=np.complex128))
    B = np.asfortranarray(np.asarray(B, dtype=np.complex128))
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    C = np.zeros((M, N), dtype=np.complex128, order="F")
    path = ctypes.c_int(0)
    ms = ctypes.c_float(0.0)
    st = lib.ttn_selftest_contract_host(A.ctypes.data_as(_D), B.ctypes.data_as(_D), C.ctypes.data_as(_D),
                                        M, N, K, int(precision), ctypes.byref(path), ctypes.byref(ms))
    if st != 0:
        raise TTNError(st, "selftest_contract_host(%d, %d, %d)" % (M, N, K))
    return C, bool(path.value), ms.value


def fp64_peak(method=0):
    """Measured FP64 rate in TFLOP/s: method 0 FMA chains (DFMA), 1 FP64
    tensor-core mma.sync m8n8k4 (DMMA)."""
    lib = load()
    out = np.zeros(1)
    st = lib.ttn_selftest_fp64_peak(int(method), _dptr(out))
    if st != 0:
        raise TTNError(st, "selftest_fp64_peak(%d)" % method)
    return float(out[0])


def svd_truncate(A, chi, eps=0.0):
    """Truncated SVD of a host complex M x N matrix (M >= N) on the device:
    returns (U (M x k), S (k), Vh (k x N), discarded weight)."""
    lib = load()
    A = np.asfortranarray(np.asarray(A, dtype=np.complex128))
    M, N = A.shape
    kmax = min(chi, N)
    U = np.zeros((M, kmax), dtype=np.complex128, order="F")
    S = np.zeros(kmax)
    Vh = np.zeros((kmax, N), dtype=np.complex128, order="F")
    k = ctypes.c_int(0)
    disc = ctypes.c_double(0.0)
    st = lib.ttn_svd_truncate(A.ctypes.data_as(_D), M, N, int(chi), float(eps), U.ctypes.data_as(_D), _dptr(S),
                              Vh.ctypes.data_as(_D), ctypes.byref(k), ctypes.byref(disc))
    if st != 0:
        raise TTNError(st, "svd_truncate(%d, %d, %d)" % (M, N, chi))
    n = k.value
    # U and Vh were written densely with k columns / rows
    Uk = U.reshape(-1, order="F")[:M * n].reshape(M, n, order="F")
    Vk = Vh.reshape(-1, order="F")[:n * N].reshape(n, N, order="F")
    return Uk, S[:n], Vk, disc.value


def inject(kind, value=0):
    """Set a fault-injection hook (INJECT_*); INJECT_NONE clears all."""
    st = load().ttn_test_inject(int(kind), int(value))
    if st != 0:
        raise TTNError(st, "test_inject(%d, %d)" % (kind, value))


def contract_split_noalloc(A_ptr, B_ptr, C_ptr, M, N, K, stream=None):
    """C = A B on device buffers (column-major complex128) without allocating;
    pointers are raw device addresses (e.g. torch tensor.data_ptr())."""
    lib = load()
    raw = getattr(stream, "cuda_stream", stream)
    st = lib.ttn_contract_split_noalloc(_P(A_ptr), _P(B_ptr), _P(C_ptr), M, N, K, _P(raw or 0))
    if st != 0:
        raise TTNError(st, "contract_split_noalloc(%d, %d, %d)" % (M, N, K))


class TTNError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


def _dptr(a):
    return a.ctypes.data_as(_D)


class TTN:
    """One TTN state on the GPU (a ``ttn_ctx``)."""

    def __init__(self, Lx, Ly, chi, levels=3):
        self.lib = load()
        h = _P()
        st = self.lib.ttn_create(Lx, Ly, levels, chi, ctypes.byref(h))
        if st != 0:
            raise TTNError(st, "ttn_create(%d, %d, %d, %d)" % (Lx, Ly, levels, chi))
        self.h = h
        self.Lx, self.Ly, self.chi, self.N = Lx, Ly, chi, Lx * Ly

    def close(self):
        if getattr(self, "h", None):
            self.lib.ttn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.ttn_last_error(self.h)
            raise TTNError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    # -- configuration -------------------------------------------------------
    def set_stream(self, stream):
        """``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.ttn_set_stream(self.h, _P(raw or 0)), "set_stream")

    def set_precision(self, p):
        self._check(self.lib.ttn_set_precision(self.h, int(p)), "set_precision")

    def set_hamiltonian(self, xy, C6, r_cut=0.0):
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(self.N, 2)
        self._check(self.lib.ttn_set_hamiltonian(self.h, _dptr(xy), float(C6), float(r_cut)),
                    "set_hamiltonian")

    def set_decay(self, gamma):
        """H - i gamma sum_i n_i (the open system of Eq. 3); 0 = closed."""
        self._check(self.lib.ttn_set_decay(self.h, float(gamma)), "set_decay")

    def apply_pulse(self, schedule):
        from .workloads import to_pulse_array
        arr = schedule if (isinstance(schedule, np.ndarray) and schedule.dtype == PULSE_DTYPE) \
            else to_pulse_array(schedule)
        arr = np.ascontiguousarray(arr)
        self._check(self.lib.ttn_apply_pulse(self.h, arr.ctypes.data_as(_P), len(arr)), "apply_pulse")

    def set_product_state(self, amps):
        a = np.ascontiguousarray(np.asarray(amps, dtype=np.complex128).reshape(self.N, 3))
        self._check(self.lib.ttn_set_product_state(self.h, a.view(np.float64).ctypes.data_as(_D)),
                    "set_product_state")

    def set_ghz(self, mask, phase=0.0):
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.int32).reshape(self.N))
        self._check(self.lib.ttn_set_ghz_target(self.h, m.ctypes.data_as(_I), float(phase)),
                    "set_ghz_target")

    # -- evolution and observables -------------------------------------------
    def step(self, dt):
        self._check(self.lib.ttn_tdvp_step(self.h, float(dt)), "tdvp_step")

    def compress_into(self, dst):
        """Truncate this state into dst (smaller bond dimension, same
        lattice): returns (sum, max) of the discarded bond weights."""
        out = np.zeros(2)
        self._check(self.lib.ttn_compress(self.h, dst.h, _dptr(out)), "compress")
        return float(out[0]), float(out[1])

    def sample(self, uniforms):
        """Projective measurement shots: uniforms (shots x N, column j = the
        j-th real atom in leaf order) -> outcomes (shots x N ints, column =
        atom id; 0: |0>, 1: |1>, 2: |r>)."""
        U = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
        if U.ndim != 2 or U.shape[1] != self.N:
            raise ValueError("uniforms must have shape (shots, %d)" % self.N)
        out = np.zeros(U.shape, dtype=np.int32)
        self._check(self.lib.ttn_sample(self.h, U.ctypes.data_as(_D), U.shape[0],
                                        out.ctypes.data_as(_I)), "sample")
        return out

    GRAD_FIELDS = {"omega_r": 0, "delta": 1}

    def fidelity_gradient(self, target, dt, n_steps, params, n_quad=6, checkpoint_every=0):
        """(F, dF/dtheta) of F = |<target|psi(t + n_steps dt)>|^2 from the
        current state; params: (schedule row, "omega_r" | "delta") pairs.
        The state and time are unchanged afterwards."""
        n = len(params)
        rows = np.ascontiguousarray([int(r) for r, _ in params], dtype=np.int32)
        fields = np.ascontiguousarray([self.GRAD_FIELDS.get(f, f) for _, f in params], dtype=np.int32)
        F = np.zeros(1)
        g = np.zeros(max(1, n))
        self._check(self.lib.ttn_fidelity_gradient(self.h, target.h, float(dt), int(n_steps), n,
                                                   rows.ctypes.data_as(_I), fields.ctypes.data_as(_I),
                                                   int(n_quad), int(checkpoint_every), _dptr(F), _dptr(g)),
                    "fidelity_gradient")
        return float(F[0]), g[:n].copy()

    def overlap(self, target):
        out = np.zeros(2)
        self._check(self.lib.ttn_overlap(self.h, target.h, _dptr(out)), "overlap")
        return complex(out[0], out[1])

    def fidelity(self, target):
        out = np.zeros(1)
        self._check(self.lib.ttn_fidelity(self.h, target.h, _dptr(out)), "fidelity")
        return float(out[0])

    def measure(self, which):
        out = np.zeros(self.N)
        self._check(self.lib.ttn_measure(self.h, int(which), _dptr(out)), "measure")
        return out

    def norm(self):
        out = np.zeros(1)
        self._check(self.lib.ttn_norm(self.h, _dptr(out)), "norm")
        return float(out[0])

    def energy(self):
        out = np.zeros(1)
        self._check(self.lib.ttn_energy(self.h, _dptr(out)), "energy")
        return float(out[0])

    def time(self):
        out = np.zeros(1)
        self._check(self.lib.ttn_get_time(self.h, _dptr(out)), "get_time")
        return float(out[0])

    def dense(self):
        out = np.zeros(2 * 3 ** self.N)
        self._check(self.lib.ttn_get_dense(self.h, _dptr(out)), "get_dense")
        return out.view(np.complex128)

    def save(self, path):
        self._check(self.lib.ttn_save(self.h, str(path).encode()), "save")

    def load(self, path):
        self._check(self.lib.ttn_load(self.h, str(path).encode()), "load")

    # -- introspection -------------------------------------------------------
    def num_nodes(self):
        n = ctypes.c_int()
        self._check(self.lib.ttn_num_nodes(self.h, ctypes.byref(n)), "num_nodes")
        return n.value

    def node_info(self, k):
        dims = (ctypes.c_int * 3)()
        ch = (ctypes.c_int * 2)()
        self._check(self.lib.ttn_node_info(self.h, k, dims, ch), "node_info")
        return tuple(dims), tuple(ch)

    def leaf_atoms(self):
        n = ctypes.c_int()
        self._check(self.lib.ttn_leaf_atoms(self.h, None, ctypes.byref(n)), "leaf_atoms")
        arr = (ctypes.c_int * n.value)()
        self._check(self.lib.ttn_leaf_atoms(self.h, arr, ctypes.byref(n)), "leaf_atoms")
        return list(arr)

    def get_node(self, k):
        """Node tensor as a (d0, d1, d2) complex array (same index meaning as
        the oracle's tensors)."""
        dims, _ = self.node_info(k)
        buf = np.zeros(2 * dims[0] * dims[1] * dims[2])
        self._check(self.lib.ttn_get_node(self.h, k, _dptr(buf)), "get_node")
        return buf.view(np.complex128).reshape(dims, order="F")

    def set_node(self, k, X):
        dims, _ = self.node_info(k)
        a = np.ascontiguousarray(np.asarray(X, dtype=np.complex128).reshape(dims).ravel(order="F"))
        self._check(self.lib.ttn_set_node(self.h, k, a.view(np.float64).ctypes.data_as(_D)), "set_node")

    def refresh_envs(self):
        self._check(self.lib.ttn_refresh_envs(self.h), "refresh_envs")

    def apply_heff(self, k, X):
        dims, _ = self.node_info(k)
        a = np.ascontiguousarray(np.asarray(X, dtype=np.complex128).reshape(dims).ravel(order="F"))
        y = np.zeros(2 * a.size)
        self._check(self.lib.ttn_apply_heff(self.h, k, a.view(np.float64).ctypes.data_as(_D), _dptr(y)),
                    "apply_heff")
        return y.view(np.complex128).reshape(dims, order="F")

    def stats(self):
        out = (ctypes.c_int64 * 6)()
        self._check(self.lib.ttn_get_stats(self.h, out), "get_stats")
        vals = list(out)
        max_err = np.array([vals[2]], dtype=np.int64).view(np.float64)[0]
        return {"krylov_runs": vals[0], "matvecs": vals[1], "max_krylov_err": float(max_err),
                "launches": vals[3], "qr_calls": vals[4], "completed_columns": vals[5]}

    PROFILE_KINDS = ("tc_gemm", "split_pack", "f64_gemm", "qr", "krylov_vectors", "elementwise")

    def profile_begin(self):
        self._check(self.lib.ttn_profile_begin(self.h), "profile_begin")

    def profile_end(self):
        out = np.zeros(4 * len(self.PROFILE_KINDS))
        self._check(self.lib.ttn_profile_end(self.h, _dptr(out), out.size), "profile_end")
        return {k: {"launches": int(out[4 * i]), "ms": out[4 * i + 1], "flops": out[4 * i + 2],
                    "bytes": out[4 * i + 3]} for i, k in enumerate(self.PROFILE_KINDS)}

    def profile_records(self):
        """(kind, M, N, K, batches, ms, flops) per launch of the last profile."""
        n = ctypes.c_int()
        self._check(self.lib.ttn_profile_records(self.h, None, 0, ctypes.byref(n)), "profile_records")
        out = np.zeros(7 * max(1, n.value))
        self._check(self.lib.ttn_profile_records(self.h, _dptr(out), n.value, ctypes.byref(n)), "profile_records")
        return out[:7 * n.value].reshape(n.value, 7)

    def reset_stats(self):
        self._check(self.lib.ttn_reset_stats(self.h), "reset_stats")
