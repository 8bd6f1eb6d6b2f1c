"""Thin ctypes binding of the C ABI in ``include/tn.h`` (same names).

Argument marshalling only: every step of the contraction runs in the
library's CUDA kernels.  Device buffers are anything with ``data_ptr()``
(torch tensors) or raw integer addresses; streams are ``torch.cuda.Stream``
objects, raw ``cudaStream_t`` integers, or None (the legacy default stream).
If the shared library is missing or fails to load, every entry point raises:
there is no fallback path.
"""

import ctypes
import os

import numpy as np

from . import builder as _build

TN_OK, TN_EINVAL, TN_ENOMEM, TN_ECUDA, TN_ETIMEOUT, TN_EUNSUPPORTED, TN_ESTATE = 0, -1, -2, -3, -4, -5, -6
TN_FP32, TN_TF32, TN_BF16X3 = 0, 1, 2
PRECISIONS = {"fp32": TN_FP32, "tf32": TN_TF32, "bf16x3": TN_BF16X3}

EXPORTS = ("tn_options_default", "tn_network", "tn_plan", "tn_plan_query", "tn_plan_widths", "tn_plan_steps",
           "tn_plan_bind", "tn_contract", "tn_contract_slices", "tn_xeb", "tn_plan_profile",
           "tn_plan_step_times", "tn_plan_set_kernel", "tn_plan_set_config", "tn_plan_set_tc_resident_b", "tn_plan_set_tc_pairs", "tn_plan_get_configs", "tn_pt_moments", "tn_pt_histogram", "tn_sample_completions",
           "tn_plan_features", "tn_plan_autotune", "tn_plan_select", "tn_mlp_grad_scratch_bytes",
           "tn_mlp_forward", "tn_mlp_grad", "tn_mlp_adam", "tn_mlp_to_half", "tn_mlp_forward_f16",
           "tn_plan_check", "tn_contract_static", "tn_fma_probe", "tn_plan_batch_slices", "tn_plan_set_chain",
           "tn_plan_get_chains", "tn_destroy", "tn_last_error")
TN_STATIC_SCRATCH_BYTES = 64 << 20
TN_PT_MAX_BINS = 8192
TN_MAX_OPEN = 16
TN_NCONFIG = 4
TN_NFEAT = TN_MLP_IN = 24
TN_MLP_HIDDEN = 128
TN_MLP_NPARAMS = TN_MLP_HIDDEN * TN_MLP_IN + TN_MLP_HIDDEN + TN_MLP_HIDDEN * TN_MLP_HIDDEN + 2 * TN_MLP_HIDDEN + 1


class TnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class tn_gate(ctypes.Structure):
    _fields_ = [("q0", ctypes.c_int32), ("q1", ctypes.c_int32), ("layer", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("m", ctypes.c_double * 32)]


class tn_circuit(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_gates", ctypes.c_int32),
                ("gates", ctypes.POINTER(tn_gate))]


class tn_options(ctypes.Structure):
    _fields_ = [("workspace_limit", ctypes.c_int64), ("slice_batch_log2", ctypes.c_int32),
                ("rescale", ctypes.c_int32), ("fuse", ctypes.c_int32), ("fuse_max_bits", ctypes.c_int32),
                ("graphs", ctypes.c_int32), ("pad0", ctypes.c_int32), ("open_mask", ctypes.c_int64),
                ("reserved", ctypes.c_int32 * 6)]


class tn_plan_info(ctypes.Structure):
    _fields_ = [("n_tensors", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("n_steps", ctypes.c_int32), ("n_unique", ctypes.c_int32), ("n_sliced", ctypes.c_int32),
                ("slice_batch_log2", ctypes.c_int32), ("n_batches", ctypes.c_int32),
                ("max_rank", ctypes.c_int32), ("n_static_steps", ctypes.c_int32),
                ("flops_ma", ctypes.c_double), ("flops_sa", ctypes.c_double), ("flops_exec", ctypes.c_double),
                ("bytes_min", ctypes.c_double), ("workspace_bytes", ctypes.c_int64),
                ("peak_tensor_bytes", ctypes.c_int64), ("upload_bytes", ctypes.c_int64),
                ("launches_per_call", ctypes.c_int64), ("n_open", ctypes.c_int32), ("n_chains", ctypes.c_int32),
                ("amps_per_row", ctypes.c_int64)]


class tn_step_info(ctypes.Structure):
    _fields_ = [("node", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32), ("mb", ctypes.c_int32),
                ("kb", ctypes.c_int32), ("nb", ctypes.c_int32), ("rank_a", ctypes.c_int32),
                ("rank_b", ctypes.c_int32), ("level", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("n_inst", ctypes.c_int64), ("n_inst_a", ctypes.c_int64), ("n_inst_b", ctypes.c_int64),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double), ("runs", ctypes.c_double),
                ("a_run_m", ctypes.c_int32), ("a_run_k", ctypes.c_int32), ("b_run_k", ctypes.c_int32),
                ("b_run_n", ctypes.c_int32), ("n_groups", ctypes.c_int64),
                ("chain", ctypes.c_int32), ("chain_last", ctypes.c_int32),
                ("c_pos_m", ctypes.c_int8 * 40), ("c_pos_n", ctypes.c_int8 * 24),
                ("max_group", ctypes.c_int64), ("n_pair_tiles", ctypes.c_int64)]


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the in-tree shared library (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path} is missing (run build())")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "tn_options_default": (None, [ctypes.POINTER(tn_options)]),
        "tn_network": (ctypes.c_int, [ctypes.POINTER(tn_circuit), vp, vp, vp, vp]),
        "tn_plan": (ctypes.c_int, [ctypes.POINTER(tn_circuit), vp, i64, vp, vp, i32,
                                   ctypes.POINTER(tn_options), ctypes.POINTER(vp)]),
        "tn_plan_query": (ctypes.c_int, [vp, ctypes.POINTER(tn_plan_info)]),
        "tn_plan_widths": (ctypes.c_int, [vp, vp, vp, vp]),
        "tn_plan_bind": (ctypes.c_int, [vp, vp, ctypes.c_size_t, vp]),
        "tn_plan_steps": (ctypes.c_int, [vp, vp, i32]),
        "tn_contract": (ctypes.c_int, [vp, ctypes.c_int, i64, i64, vp, vp]),
        "tn_contract_slices": (ctypes.c_int, [vp, ctypes.c_int, vp, i32, vp, vp]),
        "tn_xeb": (ctypes.c_int, [vp, i64, i32, vp, vp]),
        "tn_pt_moments": (ctypes.c_int, [vp, i64, i32, ctypes.c_double, vp, vp]),
        "tn_sample_completions": (ctypes.c_int, [vp, i64, i32, vp, vp, vp]),
        "tn_pt_histogram": (ctypes.c_int, [vp, i64, i32, ctypes.c_double, i32, vp, vp]),
        "tn_plan_profile": (ctypes.c_int, [vp, ctypes.c_int]),
        "tn_plan_set_kernel": (ctypes.c_int, [vp, i32, i32]),
        "tn_plan_set_config": (ctypes.c_int, [vp, i32, i32]),
        "tn_plan_set_tc_resident_b": (ctypes.c_int, [vp, i32]),
        "tn_plan_set_tc_pairs": (ctypes.c_int, [vp, i32]),
        "tn_plan_get_configs": (ctypes.c_int, [vp, vp, i32]),
        "tn_plan_features": (ctypes.c_int, [vp, ctypes.c_int, i32, vp, vp, i32]),
        "tn_plan_autotune": (ctypes.c_int, [vp, ctypes.c_int, i32, vp, vp, vp, vp]),
        "tn_plan_select": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_float, vp, ctypes.c_size_t, vp, vp]),
        "tn_mlp_grad_scratch_bytes": (ctypes.c_size_t, [i64]),
        "tn_mlp_forward": (ctypes.c_int, [vp, vp, i64, vp, vp]),
        "tn_mlp_grad": (ctypes.c_int, [vp, vp, vp, i64, vp, vp, vp, ctypes.c_size_t, vp]),
        "tn_mlp_adam": (ctypes.c_int, [vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, vp]),
        "tn_mlp_to_half": (ctypes.c_int, [vp, vp, vp]),
        "tn_mlp_forward_f16": (ctypes.c_int, [vp, vp, i64, vp, vp]),
        "tn_plan_check": (ctypes.c_int, [vp, vp]),
        "tn_contract_static": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
        "tn_fma_probe": (ctypes.c_int, [i64, i64, vp, vp]),
        "tn_plan_batch_slices": (ctypes.c_int, [vp, i64, vp, i64]),
        "tn_plan_set_chain": (ctypes.c_int, [vp, i32, i32]),
        "tn_plan_get_chains": (ctypes.c_int, [vp, vp, i32]),
        "tn_plan_step_times": (ctypes.c_int, [vp, vp, vp, i32]),
        "tn_destroy": (None, [vp]),
        "tn_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != TN_OK:
        raise TnError(rc, load().tn_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def circuit_struct(circ):
    """Marshal an ``rqc.Circuit`` into a ``tn_circuit`` (keeps the arrays alive)."""
    q0, q1, layer, m = circ.to_arrays()
    arr = (tn_gate * len(q0))()
    for i in range(len(q0)):
        arr[i].q0, arr[i].q1, arr[i].layer = int(q0[i]), int(q1[i]), int(layer[i])
        ctypes.memmove(arr[i].m, m[i].ctypes.data, 32 * 8)
    c = tn_circuit(circ.n_qubits, len(q0), arr)
    c._keep = arr
    return c


def options(**kw) -> tn_options:
    """tn_options with the library's defaults, then the given fields;
    open_qubits=[...] sets open_mask from a list of qubits."""
    o = tn_options()
    load().tn_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "open_qubits":
            k, v = "open_mask", sum(1 << int(q) for q in v)
        setattr(o, k, v)
    return o


def tn_network(circ):
    lib = load()
    c = circuit_struct(circ)
    nt, ne = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.tn_network(ctypes.byref(c), ctypes.byref(nt), ctypes.byref(ne), None, None))
    ends = np.zeros((ne.value, 2), np.int32)
    outs = np.zeros(circ.n_qubits, np.int32)
    _check(lib.tn_network(ctypes.byref(c), None, None, ends.ctypes.data, outs.ctypes.data))
    return nt.value, ne.value, ends, outs


class Plan:
    """A tn_plan handle: host planning in the constructor, device work after
    :meth:`tn_plan_bind`."""

    def __init__(self, circ, bits, tree_ssa, sliced=(), **opts):
        lib = load()
        self._lib = lib
        self.n_qubits = circ.n_qubits
        c = circuit_struct(circ)
        self._bits = np.ascontiguousarray(bits, np.uint8)
        self.k = self._bits.shape[0]
        ssa = np.ascontiguousarray(np.asarray(tree_ssa, np.int32).reshape(-1, 2))
        sl = np.ascontiguousarray(np.asarray(list(sliced), np.int32))
        o = options(**opts)
        h = ctypes.c_void_p()
        _check(lib.tn_plan(ctypes.byref(c), self._bits.ctypes.data if self.k else None, self.k,
                           ssa.ctypes.data if ssa.size else None, sl.ctypes.data if sl.size else None,
                           len(sl), ctypes.byref(o), ctypes.byref(h)))
        self.h = h.value
        self.n_sliced = len(sl)
        self._ws = None

    def __del__(self):
        if getattr(self, "h", None):
            self._lib.tn_destroy(self.h)
            self.h = None

    def tn_plan_query(self) -> dict:
        info = tn_plan_info()
        _check(self._lib.tn_plan_query(self.h, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in tn_plan_info._fields_}

    info = property(tn_plan_query)

    def tn_plan_widths(self):
        n = self.info["n_nodes"]
        w = np.zeros(n, np.int64)
        r = np.zeros(n, np.int32)
        s = np.zeros(n, np.int32)
        _check(self._lib.tn_plan_widths(self.h, w.ctypes.data, r.ctypes.data, s.ctypes.data))
        return w, r, s

    def tn_plan_steps(self):
        """Per-step features as a list of dicts (execution order)."""
        n = self.info["n_steps"]
        arr = (tn_step_info * max(n, 1))()
        _check(self._lib.tn_plan_steps(self.h, arr, n))
        out = []
        for i in range(n):
            r = {}
            for f, _ in tn_step_info._fields_:
                v = getattr(arr[i], f)
                r[f] = [x for x in v if x >= 0] if f.startswith("c_pos") else v
            out.append(r)
        return out

    def tn_plan_batch_slices(self, batch):
        """Slice ids (int64 numpy array) computed by slice batch ``batch``."""
        n = 1 << self.info["slice_batch_log2"]
        out = np.zeros(n, np.int64)
        _check(self._lib.tn_plan_batch_slices(self.h, int(batch), out.ctypes.data, n))
        return out

    def tn_plan_bind(self, workspace, nbytes=None, stream=None):
        if nbytes is None:
            nbytes = workspace.numel() * workspace.element_size()
        self._ws = workspace  # keep it alive while bound
        _check(self._lib.tn_plan_bind(self.h, _ptr(workspace), int(nbytes), _stream(stream)))

    @staticmethod
    def _check_amps(amps, n_complex, what):
        """A complex128 device buffer must hold n_complex entries (2 doubles
        each); raw integer addresses are taken on trust."""
        if hasattr(amps, "numel") and hasattr(amps, "element_size"):
            if amps.numel() * amps.element_size() < 16 * n_complex:
                raise TnError(TN_EINVAL, f"{what}: amplitude buffer holds {amps.numel() * amps.element_size()} "
                                         f"bytes, needs {16 * n_complex}")

    def tn_contract(self, amps, precision=TN_FP32, batch_lo=0, batch_hi=None, stream=None):
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self._check_amps(amps, self.k * self.info["amps_per_row"], "tn_contract")
        if batch_hi is None:
            batch_hi = self.info["n_batches"]
        _check(self._lib.tn_contract(self.h, int(precision), int(batch_lo), int(batch_hi), _ptr(amps),
                                     _stream(stream)))

    def tn_contract_slices(self, slice_ids, partials, precision=TN_FP32, stream=None):
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        ids = np.ascontiguousarray(np.asarray(slice_ids, np.int64))
        _check(self._lib.tn_contract_slices(self.h, int(precision), ids.ctypes.data, len(ids), _ptr(partials),
                                            _stream(stream)))

    def tn_contract_static(self, amps, precision=TN_FP32, stream=None):
        """Contract every slice batch into ``amps`` using the library's fixed
        device scratch instead of a bound workspace (no device allocation;
        plans above TN_STATIC_SCRATCH_BYTES are rejected)."""
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self._check_amps(amps, self.k * self.info["amps_per_row"], "tn_contract_static")
        _check(self._lib.tn_contract_static(self.h, int(precision), _ptr(amps), _stream(stream)))

    def tn_plan_set_kernel(self, step, kernel):
        _check(self._lib.tn_plan_set_kernel(self.h, int(step), int(kernel)))

    def tn_plan_set_config(self, step, config):
        _check(self._lib.tn_plan_set_config(self.h, int(step), int(config)))

    def tn_plan_set_chain(self, chain, enable):
        _check(self._lib.tn_plan_set_chain(self.h, int(chain), int(bool(enable))))

    def tn_plan_get_chains(self):
        n = self.info["n_chains"]
        c = np.zeros(max(n, 1), np.int32)
        _check(self._lib.tn_plan_get_chains(self.h, c.ctypes.data, n))
        return c[:n]

    def tn_plan_set_tc_resident_b(self, enable):
        _check(self._lib.tn_plan_set_tc_resident_b(self.h, int(bool(enable))))

    def tn_plan_set_tc_pairs(self, enable):
        _check(self._lib.tn_plan_set_tc_pairs(self.h, int(bool(enable))))

    def tn_plan_get_configs(self):
        n = self.info["n_steps"]
        c = np.zeros(max(n, 1), np.int32)
        _check(self._lib.tn_plan_get_configs(self.h, c.ctypes.data, n))
        return c[:n]

    def tn_plan_features(self, precision, config):
        """(features n_steps x TN_NFEAT float32, eligible n_steps bool) for one configuration."""
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        n = self.info["n_steps"]
        f = np.zeros((max(n, 1), TN_NFEAT), np.float32)
        e = np.zeros(max(n, 1), np.int32)
        _check(self._lib.tn_plan_features(self.h, int(precision), int(config), f.ctypes.data, e.ctypes.data, n))
        return f[:n], e[:n].astype(bool)

    def tn_plan_autotune(self, precision, amps_scratch, reps=2, step_mask=None, stream=None):
        """Exhaustive autotuner: returns ms per pass, n_steps x TN_NCONFIG (NaN: not measured)."""
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        n = self.info["n_steps"]
        t = np.full((max(n, 1), TN_NCONFIG), np.nan)
        mask = None if step_mask is None else np.ascontiguousarray(np.asarray(step_mask, np.uint8))
        _check(self._lib.tn_plan_autotune(self.h, int(precision), int(reps),
                                          None if mask is None else mask.ctypes.data, _ptr(amps_scratch),
                                          t.ctypes.data, _stream(stream)))
        return t[:n]

    def tn_plan_select(self, precision, params16, scratch, margin=0.0, stream=None):
        """Cost-model selection; returns the per-step 'uncertain' flags (bool)."""
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        n = self.info["n_steps"]
        u = np.zeros(max(n, 1), np.int32)
        nbytes = scratch.numel() * scratch.element_size()
        _check(self._lib.tn_plan_select(self.h, int(precision), _ptr(params16), float(margin), _ptr(scratch),
                                        int(nbytes), u.ctypes.data, _stream(stream)))
        return u[:n].astype(bool)

    def tn_plan_check(self, stream=None):
        _check(self._lib.tn_plan_check(self.h, _stream(stream)))

    def tn_plan_profile(self, enable=True):
        _check(self._lib.tn_plan_profile(self.h, 1 if enable else 0))

    def tn_plan_step_times(self):
        """(ms per step summed over the last call's batches, kernel family per step)."""
        n = self.info["n_steps"]
        ms = np.zeros(max(n, 1), np.float64)
        kern = np.zeros(max(n, 1), np.int32)
        _check(self._lib.tn_plan_step_times(self.h, ms.ctypes.data, kern.ctypes.data, n))
        return ms[:n], kern[:n]


def tn_xeb(amps, k, n_qubits, out, stream=None):
    _check(load().tn_xeb(_ptr(amps), int(k), int(n_qubits), _ptr(out), _stream(stream)))


def tn_sample_completions(amps, k, n_open, uniform, picks, stream=None):
    _check(load().tn_sample_completions(_ptr(amps), int(k), int(n_open), _ptr(uniform), _ptr(picks), _stream(stream)))


def tn_pt_moments(amps, k, n_qubits, fidelity, out, stream=None):
    _check(load().tn_pt_moments(_ptr(amps), int(k), int(n_qubits), float(fidelity), _ptr(out), _stream(stream)))


def tn_pt_histogram(amps, k, n_qubits, x_max, nbins, counts, stream=None):
    _check(load().tn_pt_histogram(_ptr(amps), int(k), int(n_qubits), float(x_max), int(nbins), _ptr(counts),
                                  _stream(stream)))


def tn_fma_probe(blocks, iters, out, stream=None):
    """FP32 FMA throughput probe: blocks x 256 threads x 16 x iters flops."""
    _check(load().tn_fma_probe(int(blocks), int(iters), _ptr(out), _stream(stream)))


def tn_mlp_grad_scratch_bytes(n):
    return int(load().tn_mlp_grad_scratch_bytes(int(n)))


def tn_mlp_forward(params, X, n, y, stream=None):
    _check(load().tn_mlp_forward(_ptr(params), _ptr(X), int(n), _ptr(y), _stream(stream)))


def tn_mlp_grad(params, X, t, n, grad, loss, scratch, stream=None):
    nbytes = scratch.numel() * scratch.element_size()
    _check(load().tn_mlp_grad(_ptr(params), _ptr(X), _ptr(t), int(n), _ptr(grad), _ptr(loss), _ptr(scratch),
                              int(nbytes), _stream(stream)))


def tn_mlp_adam(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().tn_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr), float(beta1),
                              float(beta2), float(eps), _stream(stream)))


def tn_mlp_to_half(params, params16, stream=None):
    _check(load().tn_mlp_to_half(_ptr(params), _ptr(params16), _stream(stream)))


def tn_mlp_forward_f16(params16, X, n, y, stream=None):
    _check(load().tn_mlp_forward_f16(_ptr(params16), _ptr(X), int(n), _ptr(y), _stream(stream)))
