"""Thin ctypes binding of libdmrgc (include/dmrgc.h): argument marshalling only.

Every function here converts Python / numpy arguments to the C types and calls
the C entry point of the same name; all compute runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built: there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libdmrgc.so")

DMRGC_FP64, DMRGC_BF16X3, DMRGC_TF32X3, DMRGC_FP32 = 0, 1, 2, 3
DMRGC_OK, DMRGC_EINVAL, DMRGC_ENOMEM, DMRGC_ECUDA, DMRGC_ENOCONV, DMRGC_ENUMERIC, DMRGC_ETIMEOUT, DMRGC_ESTATE = range(8)
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ENUMERIC",
          6: "ETIMEOUT", 7: "ESTATE"}


class DmrgcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dmrgc {STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("rows", C.c_int), ("cols", C.c_int), ("order", C.c_int)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("svd_mode", C.c_int),
                ("sweep_rel_cutoff", C.c_double), ("zip_rel_cutoff", C.c_double),
                ("max_jacobi_sweeps", C.c_int), ("seed", C.c_ulonglong),
                ("cuda_stream", C.c_void_p), ("timing", C.c_int),
                ("rsvd_oversample", C.c_int), ("rsvd_power_iters", C.c_int),
                ("rsvd_tolerance", C.c_double), ("log_rank_records", C.c_int),
                ("mpo_compress", C.c_int), ("svd_path", C.c_int)]


class Gate(C.Structure):
    _fields_ = [("q0", C.c_int), ("q1", C.c_int), ("mat", C.c_double * 32)]


class Stats(C.Structure):
    _fields_ = [("gemm_ms", C.c_double), ("gemm_flops", C.c_double), ("gemm_launches", C.c_longlong),
                ("svd_ms", C.c_double), ("svd_flops", C.c_double), ("svd_launches", C.c_longlong),
                ("jacobi_sweeps", C.c_longlong), ("mpo_ms", C.c_double),
                ("other_ms", C.c_double), ("updates", C.c_longlong), ("kernel_launches", C.c_longlong),
                ("rsvd_attempts", C.c_longlong), ("rsvd_accepted", C.c_longlong),
                ("eig_svds", C.c_longlong), ("eig_fallbacks", C.c_longlong), ("eig_skipped", C.c_longlong)]


class BatchItem(C.Structure):
    _fields_ = [("rows", C.c_int), ("cols", C.c_int), ("grid_view", Grid), ("chi", C.c_int),
                ("n_layers", C.c_int), ("n_sweeps", C.c_int), ("gates", C.POINTER(Gate)),
                ("layer_sizes", C.POINTER(C.c_int)), ("log_F_tilde", C.c_double),
                ("seconds", C.c_double), ("updates", C.c_longlong), ("status", C.c_int),
                ("worker", C.c_int)]


_lib = None


def lib():
    """Load libdmrgc.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libdmrgc.so not built at {_LIB_PATH}; run "
                              "`python -m paper_2207_05612_gb300.build`")
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER
        L.dmrgc_default_options.argtypes = [P(Options)]
        L.dmrgc_create.argtypes = [C.c_int, P(Grid), C.c_int, P(Options), P(C.c_void_p)]
        L.dmrgc_create_grouped.argtypes = [C.c_int, P(Grid), C.c_void_p, C.c_int, C.c_int, P(Options),
                                           P(C.c_void_p)]
        L.dmrgc_group_sizes.argtypes = [C.c_void_p, C.c_void_p, P(C.c_int)]
        L.dmrgc_metropolis.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_ulonglong, C.c_void_p,
                                       P(C.c_longlong)]
        L.dmrgc_apply_layer.argtypes = [C.c_void_p, P(Gate), C.c_int]
        L.dmrgc_sweep.argtypes = [C.c_void_p, C.c_int, P(C.c_double)]
        L.dmrgc_fidelity.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double)]
        L.dmrgc_amplitude.argtypes = [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]
        L.dmrgc_sample.argtypes = [C.c_void_p, C.c_longlong, C.c_ulonglong, C.c_void_p]
        L.dmrgc_bond_dims.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.dmrgc_mps_size.argtypes = [C.c_void_p]
        L.dmrgc_mps_size.restype = C.c_longlong
        L.dmrgc_get_mps.argtypes = [C.c_void_p, C.c_void_p, P(C.c_int)]
        L.dmrgc_step_history.argtypes = [C.c_void_p, C.c_void_p, C.c_int, P(C.c_int)]
        L.dmrgc_get_stats.argtypes = [C.c_void_p, P(Stats)]
        L.dmrgc_reset_stats.argtypes = [C.c_void_p]
        L.dmrgc_last_error.argtypes = [C.c_void_p]
        L.dmrgc_last_error.restype = C.c_char_p
        L.dmrgc_destroy.argtypes = [C.c_void_p]
        L.dmrgc_destroy.restype = None
        L.dmrgc_test_gemm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_void_p, C.c_longlong, C.c_longlong, C.c_void_p,
                                      C.c_longlong, C.c_longlong, C.c_void_p]
        L.dmrgc_test_svd.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_double,
                                     C.c_void_p, P(C.c_int), C.c_void_p]
        L.dmrgc_test_svd_gram.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_double,
                                          C.c_void_p, P(C.c_int), C.c_void_p]
        L.dmrgc_svd_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_double,
                                        C.c_void_p, P(C.c_int), C.c_void_p, C.c_void_p]
        L.dmrgc_batch_run.argtypes = [P(BatchItem), C.c_int, C.c_int, P(Options), C.c_void_p, P(C.c_double)]
        L.dmrgc_set_jacobi_kernel.argtypes = [C.c_int]
        L.dmrgc_set_wait_limit.argtypes = [C.c_ulonglong]
        L.dmrgc_set_mps.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double]
        L.dmrgc_sweep_updates.argtypes = [C.c_void_p, C.c_longlong, P(C.c_double)]
        L.dmrgc_overlap.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.dmrgc_xeb.argtypes = [C.c_void_p, C.c_void_p, C.c_longlong, C.c_ulonglong, P(C.c_double),
                                P(C.c_double)]
        L.dmrgc_overlap_layer.argtypes = [C.c_void_p, C.c_void_p, P(Gate), C.c_int, C.c_void_p]
        fp = C.c_void_p
        L.dmrgc_set_rank_model.argtypes = [C.c_void_p, fp]
        L.dmrgc_rank_records.argtypes = [C.c_void_p, fp, fp, C.c_int, P(C.c_int)]
        L.dmrgc_mlp_train.argtypes = [fp, fp, C.c_int, C.c_int, C.c_int, C.c_float, C.c_ulonglong, fp, fp]
        L.dmrgc_mlp_loss_grad.argtypes = [fp, fp, fp, C.c_int, P(C.c_float), fp]
        L.dmrgc_mlp_predict.argtypes = [fp, fp, C.c_int, C.c_int, fp]
        for name in ("dmrgc_metropolis", "dmrgc_create_grouped", "dmrgc_group_sizes", "dmrgc_set_mps", "dmrgc_sweep_updates", "dmrgc_set_wait_limit", "dmrgc_xeb", "dmrgc_overlap", "dmrgc_overlap_layer", "dmrgc_set_jacobi_kernel", "dmrgc_set_rank_model", "dmrgc_rank_records", "dmrgc_mlp_train",
                     "dmrgc_mlp_loss_grad", "dmrgc_mlp_predict", "dmrgc_batch_run", "dmrgc_svd_noalloc", "dmrgc_test_gemm", "dmrgc_test_svd", "dmrgc_test_svd_gram", "dmrgc_default_options", "dmrgc_create", "dmrgc_apply_layer", "dmrgc_sweep",
                     "dmrgc_fidelity", "dmrgc_amplitude", "dmrgc_sample", "dmrgc_bond_dims",
                     "dmrgc_get_mps", "dmrgc_step_history", "dmrgc_get_stats", "dmrgc_reset_stats"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(status: int, ctx=None):
    if status != 0:
        msg = lib().dmrgc_last_error(ctx).decode() if ctx else ""
        raise DmrgcError(status, msg)


def pack_gates(layer) -> "C.Array":
    """[(q0, q1, U)] -> array of dmrgc_gate (row-major complex128, re/im interleaved)."""
    arr = (Gate * max(len(layer), 1))()
    for i, (q0, q1, u) in enumerate(layer):
        flat = np.asarray(u, dtype=np.complex128).reshape(-1)
        buf = np.zeros(32)
        buf[0:2 * flat.size:2] = flat.real
        buf[1:2 * flat.size:2] = flat.imag
        arr[i].q0 = int(q0)
        arr[i].q1 = int(q1)
        arr[i].mat[:] = buf.tolist()
    return arr


def dmrgc_default_options() -> Options:
    o = Options()
    _check(lib().dmrgc_default_options(C.byref(o)))
    return o


ORDERS = {"V": 0, "H": 1, "D": 2}   # chain orders: columns, rows, anti-diagonals


def dmrgc_create(n_qubits: int, rows: int, cols: int, chi: int, options: Options | None = None,
                 order: int = 0, groups=None):
    """groups: None (one qubit per tensor, two-site updates) or the sites per
    tensor (single-site updates over grouped qubits)."""
    g = Grid(rows, cols, order)
    h = C.c_void_p()
    opt = options if options is not None else dmrgc_default_options()
    if groups is None:
        _check(lib().dmrgc_create(n_qubits, C.byref(g), chi, C.byref(opt), C.byref(h)))
    else:
        gs = np.ascontiguousarray(groups, dtype=np.int32)
        _check(lib().dmrgc_create_grouped(n_qubits, C.byref(g), gs.ctypes.data, len(gs), chi, C.byref(opt),
                                          C.byref(h)))
    return h


def dmrgc_group_sizes(ctx) -> list[int]:
    n = C.c_int()
    _check(lib().dmrgc_group_sizes(ctx, None, C.byref(n)), ctx)
    out = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(lib().dmrgc_group_sizes(ctx, out.ctypes.data, C.byref(n)), ctx)
    return out[:n.value].tolist()


def dmrgc_apply_layer(ctx, layer) -> None:
    gates = pack_gates(layer)
    _check(lib().dmrgc_apply_layer(ctx, gates, len(layer)), ctx)


def dmrgc_sweep(ctx, n_sweeps: int) -> float:
    f = C.c_double()
    _check(lib().dmrgc_sweep(ctx, n_sweeps, C.byref(f)), ctx)
    return f.value


def dmrgc_fidelity(ctx) -> tuple[float, float]:
    lf, fd = C.c_double(), C.c_double()
    _check(lib().dmrgc_fidelity(ctx, C.byref(lf), C.byref(fd)), ctx)
    return lf.value, fd.value


def dmrgc_amplitude(ctx, bits: np.ndarray) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    out = np.zeros((bits.shape[0], 2), dtype=np.float64)
    _check(lib().dmrgc_amplitude(ctx, bits.ctypes.data, bits.shape[0], out.ctypes.data), ctx)
    return out[:, 0] + 1j * out[:, 1]


def dmrgc_sample(ctx, count: int, seed: int, n_qubits: int) -> np.ndarray:
    out = np.zeros((count, n_qubits), dtype=np.uint8)
    _check(lib().dmrgc_sample(ctx, count, C.c_ulonglong(seed), out.ctypes.data), ctx)
    return out


def dmrgc_metropolis(ctx, chains: int, steps: int, seed: int, n_qubits: int):
    out = np.zeros((chains, steps, n_qubits), dtype=np.uint8)
    acc = C.c_longlong()
    _check(lib().dmrgc_metropolis(ctx, chains, steps, C.c_ulonglong(seed), out.ctypes.data, C.byref(acc)), ctx)
    return out, acc.value


def dmrgc_bond_dims(ctx, n_qubits: int) -> tuple[list[int], list[int]]:
    a = np.zeros(max(n_qubits - 1, 1), dtype=np.int32)
    b = np.zeros(max(n_qubits - 1, 1), dtype=np.int32)
    _check(lib().dmrgc_bond_dims(ctx, a.ctypes.data, b.ctypes.data), ctx)
    return a[:n_qubits - 1].tolist(), b[:n_qubits - 1].tolist()


def dmrgc_get_mps(ctx, n_qubits: int) -> tuple[list[np.ndarray], int]:
    size = lib().dmrgc_mps_size(ctx)
    buf = np.zeros(2 * size, dtype=np.float64)
    centre = C.c_int()
    _check(lib().dmrgc_get_mps(ctx, buf.ctypes.data, C.byref(centre)), ctx)
    sizes = dmrgc_group_sizes(ctx)
    bonds, _ = dmrgc_bond_dims(ctx, n_qubits)
    chis = [1] + bonds[:len(sizes) - 1] + [1]
    z = buf[0::2] + 1j * buf[1::2]
    out, off = [], 0
    for i, r in enumerate(sizes):
        n = chis[i] * 2 ** r * chis[i + 1]
        out.append(z[off:off + n].reshape(chis[i], 2 ** r, chis[i + 1]))
        off += n
    return out, centre.value


def dmrgc_set_mps(ctx, mps, log_ft: float = 0.0) -> None:
    """Load an MPS (list of [chi_l, 2, chi_r] arrays, the layout of
    dmrgc_get_mps) as the state the next apply_layer compresses."""
    bonds = np.array([mps[0].shape[0]] + [a.shape[2] for a in mps], dtype=np.int32)
    flat = np.concatenate([np.ascontiguousarray(a, dtype=np.complex128).reshape(-1) for a in mps])
    _check(lib().dmrgc_set_mps(ctx, flat.ctypes.data, bonds.ctypes.data, float(log_ft)), ctx)


def dmrgc_sweep_updates(ctx, n_updates: int) -> float:
    f = C.c_double()
    _check(lib().dmrgc_sweep_updates(ctx, int(n_updates), C.byref(f)), ctx)
    return f.value


def dmrgc_step_history(ctx) -> list[float]:
    n = C.c_int()
    _check(lib().dmrgc_step_history(ctx, None, 0, C.byref(n)), ctx)
    f = np.zeros(max(n.value, 1))
    _check(lib().dmrgc_step_history(ctx, f.ctypes.data, n.value, C.byref(n)), ctx)
    return f[:n.value].tolist()


def dmrgc_get_stats(ctx) -> dict:
    s = Stats()
    _check(lib().dmrgc_get_stats(ctx, C.byref(s)), ctx)
    return {name: getattr(s, name) for name, _ in Stats._fields_}


def dmrgc_reset_stats(ctx) -> None:
    _check(lib().dmrgc_reset_stats(ctx), ctx)


def dmrgc_destroy(ctx) -> None:
    if ctx:
        lib().dmrgc_destroy(ctx)


def dmrgc_test_gemm(precision: int, a: np.ndarray, b: np.ndarray, op_a: int, op_b: int,
                    m: int, n: int, k: int) -> np.ndarray:
    """C = op(A) op(B) on the device (diagnostic entry point)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    out = np.zeros((m, n), dtype=np.complex128)
    _check(lib().dmrgc_test_gemm(precision, m, n, k, op_a, op_b, a.ctypes.data, a.size, a.shape[1],
                                 b.ctypes.data, b.size, b.shape[1], out.ctypes.data))
    return out


def dmrgc_test_svd(precision: int, g: np.ndarray, chi: int, rel_cut: float):
    """Jacobi SVD + truncation of g (m x n) on the device (diagnostic entry point).
    Returns (s, k, U_k)."""
    m, n = g.shape
    gc = np.asfortranarray(g, dtype=np.complex128)
    s = np.zeros(n)
    k = C.c_int()
    u = np.zeros((m, n), dtype=np.complex128)
    _check(lib().dmrgc_test_svd(precision, m, n, gc.ctypes.data, chi, rel_cut, s.ctypes.data,
                                C.byref(k), u.ctypes.data))
    kk = k.value
    return s, kk, u.reshape(-1)[:m * kk].reshape(m, kk)


def dmrgc_test_svd_gram(precision: int, g: np.ndarray, chi: int, rel_cut: float):
    """Gram-eigensolver truncated SVD of g (m x n) on the device (diagnostic
    entry point).  Returns (s, k, U_k); k = -1 and U_k = None when the kept
    eigenvalues are not resolved."""
    m, n = g.shape
    gc = np.asfortranarray(g, dtype=np.complex128)
    s = np.zeros(m)
    k = C.c_int()
    u = np.zeros((m, chi), dtype=np.complex128)
    _check(lib().dmrgc_test_svd_gram(precision, m, n, gc.ctypes.data, chi, rel_cut, s.ctypes.data,
                                     C.byref(k), u.ctypes.data))
    kk = k.value
    if kk < 0:
        return s, kk, None
    return s, kk, u.reshape(-1)[:m * kk].reshape(m, kk)


def dmrgc_svd_noalloc(precision: int, g_ptr: int, m: int, n: int, chi: int, rel_cut: float,
                      s_ptr: int, u_ptr: int, stream: int = 0) -> int:
    """Truncated SVD of a device matrix without any allocation (device
    pointers in and out; see include/dmrgc.h).  Returns k."""
    k = C.c_int()
    _check(lib().dmrgc_svd_noalloc(precision, m, n, C.c_void_p(g_ptr), chi, rel_cut,
                                   C.c_void_p(s_ptr), C.byref(k), C.c_void_p(u_ptr),
                                   C.c_void_p(stream)))
    return k.value


def pack_batch(instances):
    """[(rows, cols, chi, layers, n_sweeps)] -> (array of dmrgc_batch_item, keep-alive list).
    `layers` is a list of gate lists [(q0, q1, U)]."""
    items = (BatchItem * max(len(instances), 1))()
    keep = []
    for i, (rows, cols, chi, layers, n_sweeps) in enumerate(instances):
        flat = [g for layer in layers for g in layer]
        gates = pack_gates(flat)
        sizes = (C.c_int * max(len(layers), 1))(*[len(layer) for layer in layers])
        keep += [gates, sizes]
        it = items[i]
        it.rows, it.cols, it.chi = rows, cols, chi
        it.grid_view = Grid(rows, cols, 0)
        it.n_layers, it.n_sweeps = len(layers), n_sweeps
        it.gates = C.cast(gates, C.POINTER(Gate))
        it.layer_sizes = C.cast(sizes, C.POINTER(C.c_int))
        it.status = -1
    return items, keep


def dmrgc_batch_run(items, count: int, n_workers: int, options: Options | None = None,
                    rank_model: np.ndarray | None = None) -> float:
    """Runs `count` packed instances on `n_workers` streams; fills the items'
    outputs and returns the wall time in seconds.  rank_model: parameters for
    svd_mode 2 (loaded into every worker's context)."""
    wall = C.c_double()
    opt = options if options is not None else dmrgc_default_options()
    model = None if rank_model is None else _f32(rank_model, (MLP_PARAMS,))
    _check(lib().dmrgc_batch_run(items, count, n_workers, C.byref(opt),
                                 None if model is None else model.ctypes.data, C.byref(wall)))
    return wall.value


MLP_IN, MLP_HIDDEN = 36, 128
MLP_PARAMS = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN + 1


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def dmrgc_set_rank_model(ctx, params: np.ndarray) -> None:
    p = _f32(params, (MLP_PARAMS,))
    _check(lib().dmrgc_set_rank_model(ctx, p.ctypes.data), ctx)


def dmrgc_rank_records(ctx, max_records: int = 1 << 20):
    """Moves the logged (inputs [n][36], labels [n]) out of the context."""
    cnt = C.c_int()
    x = np.zeros((max_records, MLP_IN), dtype=np.float32)
    y = np.zeros(max_records, dtype=np.float32)
    _check(lib().dmrgc_rank_records(ctx, x.ctypes.data, y.ctypes.data, max_records, C.byref(cnt)), ctx)
    return x[:cnt.value].copy(), y[:cnt.value].copy()


def dmrgc_mlp_train(x: np.ndarray, y: np.ndarray, epochs: int, batch: int = 256, lr: float = 1e-3,
                    seed: int = 0):
    """Train the rank model on the GPU; returns (params, per-epoch loss)."""
    x = _f32(x)
    y = _f32(y)
    n = y.size
    assert x.shape == (n, MLP_IN)
    params = np.zeros(MLP_PARAMS, dtype=np.float32)
    loss = np.zeros(epochs, dtype=np.float32)
    _check(lib().dmrgc_mlp_train(x.ctypes.data, y.ctypes.data, n, epochs, batch, lr, seed,
                                 params.ctypes.data, loss.ctypes.data))
    return params, loss


def dmrgc_mlp_loss_grad(params: np.ndarray, x: np.ndarray, y: np.ndarray):
    p = _f32(params, (MLP_PARAMS,))
    x = _f32(x)
    y = _f32(y)
    loss = C.c_float()
    grad = np.zeros(MLP_PARAMS, dtype=np.float32)
    _check(lib().dmrgc_mlp_loss_grad(p.ctypes.data, x.ctypes.data, y.ctypes.data, y.size, C.byref(loss),
                                     grad.ctypes.data))
    return loss.value, grad


def dmrgc_mlp_predict(params: np.ndarray, x: np.ndarray, bf16: bool = True) -> np.ndarray:
    p = _f32(params, (MLP_PARAMS,))
    x = _f32(x)
    out = np.zeros(x.shape[0], dtype=np.float32)
    _check(lib().dmrgc_mlp_predict(p.ctypes.data, x.ctypes.data, x.shape[0], 1 if bf16 else 0,
                                   out.ctypes.data))
    return out


def dmrgc_overlap(ctx_a, ctx_b) -> complex:
    """<a|b> of the two contexts' current states."""
    out = np.zeros(2)
    _check(lib().dmrgc_overlap(ctx_a, ctx_b, out.ctypes.data), ctx_a)
    return complex(out[0], out[1])


def dmrgc_overlap_layer(ctx_a, ctx_b, gates) -> complex:
    """<a| U |b> with U the given gates (one exact MPO)."""
    packed = pack_gates(gates)
    out = np.zeros(2)
    _check(lib().dmrgc_overlap_layer(ctx_a, ctx_b, packed, len(gates), out.ctypes.data), ctx_a)
    return complex(out[0], out[1])


def dmrgc_xeb(ctx_sampled, ctx_reference, count: int, seed: int) -> tuple[float, float]:
    """(F_B, standard error) of `count` samples of one context scored by the other."""
    fb, se = C.c_double(), C.c_double()
    _check(lib().dmrgc_xeb(ctx_sampled, ctx_reference, count, seed, C.byref(fb), C.byref(se)), ctx_sampled)
    return fb.value, se.value


def dmrgc_set_jacobi_kernel(variant: int) -> None:
    """0: column-pair Jacobi kernel (default); 1: Gram-block kernel."""
    _check(lib().dmrgc_set_jacobi_kernel(int(variant)))


def dmrgc_set_wait_limit(spins: int) -> None:
    """Iteration limit of the Jacobi kernels' spin waits on the current device (0 = default)."""
    _check(lib().dmrgc_set_wait_limit(int(spins)))


class Context:
    """Owning handle around the C context (marshalling only)."""

    def __init__(self, rows: int, cols: int, chi: int, precision: int = DMRGC_FP64,
                 timing: bool = False, stream=None, order: str = "V", groups=None, **opts):
        o = dmrgc_default_options()
        o.precision = precision
        o.timing = 1 if timing else 0
        if stream is not None:
            o.cuda_stream = C.c_void_p(int(stream))
        for k, v in opts.items():
            setattr(o, k, v)
        self.n = rows * cols
        self.h = dmrgc_create(self.n, rows, cols, chi, o, ORDERS[order], groups)

    def apply_layer(self, layer):
        dmrgc_apply_layer(self.h, layer)

    def sweep(self, n_sweeps: int = 2) -> float:
        return dmrgc_sweep(self.h, n_sweeps)

    def fidelity(self):
        return dmrgc_fidelity(self.h)

    def amplitude(self, bits):
        return dmrgc_amplitude(self.h, bits)

    def sample(self, count: int, seed: int):
        return dmrgc_sample(self.h, count, seed, self.n)

    def metropolis(self, chains: int, steps: int, seed: int):
        return dmrgc_metropolis(self.h, chains, steps, seed, self.n)

    def bond_dims(self):
        return dmrgc_bond_dims(self.h, self.n)

    def get_mps(self):
        return dmrgc_get_mps(self.h, self.n)

    def set_mps(self, mps, log_ft: float = 0.0):
        dmrgc_set_mps(self.h, mps, log_ft)

    def sweep_updates(self, n_updates: int) -> float:
        return dmrgc_sweep_updates(self.h, n_updates)

    def history(self):
        return dmrgc_step_history(self.h)

    def stats(self):
        return dmrgc_get_stats(self.h)

    def reset_stats(self):
        dmrgc_reset_stats(self.h)

    def set_rank_model(self, params):
        dmrgc_set_rank_model(self.h, params)

    def rank_records(self):
        return dmrgc_rank_records(self.h)

    def overlap(self, other: "Context", gates=None) -> complex:
        """<self|other> of the two current states, or <self| U |other> with
        U the given gates."""
        if gates is None:
            return dmrgc_overlap(self.h, other.h)
        return dmrgc_overlap_layer(self.h, other.h, gates)

    def close(self):
        if self.h:
            dmrgc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
