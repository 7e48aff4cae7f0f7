"""Python binding of the Squint C ABI (include/squint.h): argument marshalling only.

Every step of the update and of inference runs in libsquint.so's CUDA kernels.
There is no CPU or PyTorch fallback: if the library is missing or fails to
load, every entry point raises.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsquint.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EAGAIN, ESTATE = 0, -1, -2, -3, -4, -5, -6
PREC_FP32, PREC_BF16, PREC_FP8, PREC_MXFP8 = 0, 1, 2, 3
MAX_CONV, MAX_HIDDEN = 8, 4


class SquintError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {code} ({_strerror(code)}) {_last_error()}")


class Config(ctypes.Structure):
    _fields_ = [
        ("obs_c", ctypes.c_int32), ("obs_h", ctypes.c_int32), ("obs_w", ctypes.c_int32),
        ("squint_f", ctypes.c_int32), ("shift_pad", ctypes.c_int32),
        ("proprio_dim", ctypes.c_int32), ("action_dim", ctypes.c_int32),
        ("conv_layers", ctypes.c_int32), ("conv_ch", ctypes.c_int32),
        ("conv_stride", ctypes.c_int32 * MAX_CONV),
        ("proj_dim", ctypes.c_int32), ("n_hidden", ctypes.c_int32),
        ("hidden", ctypes.c_int32 * MAX_HIDDEN),
        ("n_critics", ctypes.c_int32), ("atoms", ctypes.c_int32), ("batch", ctypes.c_int32),
        ("policy_freq", ctypes.c_int32), ("precision", ctypes.c_int32), ("max_k", ctypes.c_int32),
        ("critic_kind", ctypes.c_int32), ("cdq", ctypes.c_int32), ("recompute_chunk", ctypes.c_int32),
        ("v_min", ctypes.c_double), ("v_max", ctypes.c_double), ("gamma", ctypes.c_double),
        ("lr", ctypes.c_double), ("tau", ctypes.c_double), ("init_alpha", ctypes.c_double),
        ("target_entropy", ctypes.c_double), ("ln_eps", ctypes.c_double),
        ("log_std_min", ctypes.c_double), ("log_std_max", ctypes.c_double),
        ("adam_b1", ctypes.c_double), ("adam_b2", ctypes.c_double), ("adam_eps", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class Replay(ctypes.Structure):
    _fields_ = [("obs", ctypes.c_void_p), ("proprio", ctypes.c_void_p), ("action", ctypes.c_void_p),
                ("reward", ctypes.c_void_p), ("done", ctypes.c_void_p), ("n", ctypes.c_int64)]


class UpdateStats(ctypes.Structure):
    _fields_ = [("critic_loss", ctypes.c_float), ("actor_loss", ctypes.c_float), ("alpha_loss", ctypes.c_float),
                ("alpha", ctypes.c_float), ("q_mean", ctypes.c_float), ("entropy", ctypes.c_float),
                ("update_idx", ctypes.c_int64)]


class PinnedStats:
    """Page-locked host room for the statistics of k updates: the buffer squint_update_async
    fills from the stream (read it once the stream has passed that call)."""

    def __init__(self, k):
        import torch
        self.k = int(k)
        self._buf = torch.empty(self.k * ctypes.sizeof(UpdateStats), dtype=torch.uint8, pin_memory=True)
        self._arr = (UpdateStats * self.k).from_address(self._buf.data_ptr())

    @property
    def ptr(self):
        return self._buf.data_ptr()

    def read(self):
        return [{f: getattr(s, f) for f, _ in UpdateStats._fields_} for s in self._arr]


class ServeResult(ctypes.Structure):
    _fields_ = [("latency_us", ctypes.c_double), ("policy_version", ctypes.c_int64),
                ("device_begin_us", ctypes.c_double), ("device_end_us", ctypes.c_double),
                ("slot", ctypes.c_int32), ("batch_rows", ctypes.c_int32)]


class ActRequest(ctypes.Structure):
    _fields_ = [("group_id", ctypes.c_uint64), ("n", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("rng_key", ctypes.c_uint64), ("obs", ctypes.c_void_p), ("proprio", ctypes.c_void_p),
                ("actions", ctypes.c_void_p)]


_lib = None


def load():
    """Load libsquint.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2602_21203_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, U64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    sig = {
        "squint_config_preset": (I, [ctypes.c_char_p, P]),
        "squint_param_count": (I64, [P]),
        "squint_create": (I, [P, P, ctypes.POINTER(P)]),
        "squint_set_replay": (I, [P, P]),
        "squint_destroy": (I, [P]),
        "squint_update": (I, [P, I, P, P]),
        "squint_update_eager": (I, [P, I, P, P]),
        "squint_update_async": (I, [P, I, P, P]),
        "squint_update_check": (I, [P, P]),
        "squint_act": (I, [P, P, I, P]),
        "squint_refresh_policy": (I, [P, P]),
        "squint_serve_start": (I, [P, I, SZ]),
        "squint_serve_submit": (I, [P, P, ctypes.POINTER(U64)]),
        "squint_serve_poll": (I, [P, U64, I64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)]),
        "squint_serve_poll_ex": (I, [P, U64, I64, P]),
        "squint_serve_info": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I64)]),
        "squint_serve_stop": (I, [P]),
        "squint_get_params": (I, [P, P, I64]),
        "squint_set_params": (I, [P, P, I64]),
        "squint_get_state": (I, [P, P, ctypes.POINTER(SZ)]),
        "squint_set_state": (I, [P, P, SZ]),
        "squint_debug_tensor": (I, [P, ctypes.c_char_p, P, ctypes.POINTER(SZ)]),
        "squint_set_debug": (I, [P, ctypes.c_char_p, I64]),
        "squint_struct_size": (SZ, [ctypes.c_char_p]),
        "squint_graph_kernel_count": (I64, [P, I]),
        "squint_device_bytes": (I64, [P]),
        "squint_profile_update": (I, [P, P, I, ctypes.POINTER(I), P]),
        "squint_phase_name": (ctypes.c_char_p, [I]),
        "squint_profile_kernels": (I, [P, I, P, P, P, P, P, ctypes.POINTER(I), P]),
        "squint_trace_update": (I, [P, I, P, P, P, P, ctypes.POINTER(I), P]),
        "squint_op_gemm": (I, [I, I, I, I, P, I64, I64, P, I64, I64, P, I64, P, I, P]),
        "squint_op_relu_bwd": (I, [I, I64, P, P, P, P]),
        "squint_op_squint_store": (I, [I, I, I, I, I, P, P, I64, I64, P]),
        "squint_op_gemm_fp8_workspace": (SZ, [I, I, I]),
        "squint_op_cast_bf16": (I, [I, I, P, I64, P, I64, P]),
        "squint_op_mlp_bwd_bf16": (I, [I, I, I, I, I, P, I64, P, P, P, P, P, P, P, P, P, P, I, I, P, I64, P]),
        "squint_op_mlp_bf16": (I, [I, I, I, I, I, P, I64, P, P, P, P, P, ctypes.c_float, P, I64, P, P, P, P, P, I, P]),
        "squint_op_gemm_layernorm": (I, [I, I, I, P, I64, P, I64, P, P, P, ctypes.c_float, I, P, P, P, P, P, P]),
        "squint_op_gemm_fp8": (I, [I, I, I, P, I64, P, I64, P, I64, P, P, SZ, P]),
        "squint_op_mx_scale_bytes": (I64, [I, I]),
        "squint_op_quantize_mxfp8": (I, [I, I, P, I64, P, I64, P, P]),
        "squint_op_gemm_mxfp8": (I, [I, I, I, P, I64, P, P, I64, P, P, I64, P, P]),
        "squint_op_conv3x3_fwd": (I, [I, I, I, I, I, I, I, P, P, P, P, I, P]),
        "squint_op_conv3x3_workspace": (SZ, [I, I, I, I, I, I, I]),
        "squint_op_conv3x3_bwd": (I, [I, I, I, I, I, I, I, P, P, P, P, P, P, P, P, SZ, P]),
        "squint_op_layernorm_fwd": (I, [I, I, P, P, P, ctypes.c_float, I, P, P, P, P]),
        "squint_op_layernorm_bwd": (I, [I, I, P, P, P, P, P, P, P, P, P, P]),
        "squint_op_categorical_ce": (I, [I, I, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float, P, P, P, P]),
        "squint_op_c51_project": (I, [I, I, I, P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_float, P, P]),
        "squint_op_tanh_gaussian_fwd": (I, [I, I, P, P, ctypes.c_float, ctypes.c_float, P, P, P]),
        "squint_op_tanh_gaussian_bwd": (I, [I, I, P, P, P, P, ctypes.c_float, ctypes.c_float, P, P]),
        "squint_op_to_phwc": (I, [I, I, I, P, P, P]),
        "squint_op_from_phwc": (I, [I, I, I, P, P, P]),
        "squint_op_conv32_layouts": (I, [P, P, P, P]),
        "squint_op_conv32": (I, [I, I, I, I, P, P, P, I, P, P, P, P]),
        "squint_op_conv0_bf16": (I, [I, I, I, I, I, P, P, P, P, P]),
        "squint_op_wgrad32_workspace": (SZ, [I]),
        "squint_op_wgrad32": (I, [I, I, I, P, P, P, P, P, SZ, P]),
        "squint_op_conv3x3_wgrad_noalloc_max": (I64, []),
        "squint_op_conv3x3_wgrad_noalloc": (I, [I, I, I, I, I, I, P, P, P, P, P]),
        "squint_strerror": (ctypes.c_char_p, [I]),
        "squint_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    for cname, cls in (("squint_config", Config), ("squint_replay", Replay), ("squint_update_stats", UpdateStats),
                       ("squint_act_request", ActRequest)):
        if lib.squint_struct_size(cname.encode()) != ctypes.sizeof(cls):
            raise RuntimeError(f"{cname}: binding layout does not match libsquint.so")
    _lib = lib
    return lib


def exported_symbols():
    """Names the header declares that the loaded library exports."""
    lib = load()
    return [n for n in dir(lib) if n.startswith("squint_")]


def _strerror(code):
    return load().squint_strerror(code).decode()


def _last_error():
    return load().squint_last_error().decode()


def _check(code, what):
    if code != OK:
        raise SquintError(code, what)


def _ptr(t):
    return ctypes.c_void_p(None if t is None else t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_config(cfg, precision=PREC_FP32, max_k=None):
    """squint_config from a workload dict (keys as in paper_2602_21203_gb300.synth)."""
    c = Config()
    for k in ("obs_c", "obs_h", "obs_w", "squint_f", "shift_pad", "proprio_dim", "action_dim", "conv_layers",
              "conv_ch", "proj_dim", "n_critics", "atoms", "batch", "policy_freq"):
        setattr(c, k, int(cfg[k]))
    strides = (cfg.get("conv_strides") or [2] + [1] * (cfg["conv_layers"] - 1)) if cfg["conv_layers"] > 0 else []
    for i, s in enumerate(strides):
        c.conv_stride[i] = int(s)
    c.n_hidden = len(cfg["hidden"])
    for i, h in enumerate(cfg["hidden"]):
        c.hidden[i] = int(h)
    c.precision = int(precision)
    c.max_k = int(max_k if max_k is not None else max(8, cfg.get("utd", 1)))
    c.recompute_chunk = int(cfg.get("recompute_chunk", 0))
    c.critic_kind = 1 if cfg.get("critic", "c51") == "mse" else 0
    c.cdq = 1 if cfg.get("cdq", False) else 0
    for k in ("v_min", "v_max", "gamma", "lr", "tau", "init_alpha", "ln_eps", "log_std_min", "log_std_max",
              "adam_b1", "adam_b2", "adam_eps"):
        setattr(c, k, float(cfg[k]))
    te = cfg.get("target_entropy")
    c.target_entropy = math.nan if te is None else float(te)
    c.seed = int(cfg["seed"])
    return c


def param_count(cfg):
    n = load().squint_param_count(ctypes.byref(make_config(cfg)))
    if n < 0:
        raise SquintError(EINVAL, "squint_param_count")
    return int(n)


class Learner:
    """One learner handle (squint_create ... squint_destroy) on the current CUDA device."""

    def __init__(self, cfg, ring=None, precision=PREC_FP32, max_k=None):
        self.lib = load()
        self.cfg = cfg
        self.c = make_config(cfg, precision, max_k)
        self.h = ctypes.c_void_p()
        self._ring = None
        rp = None
        if ring is not None:
            rp = ctypes.byref(self._replay(ring))
        _check(self.lib.squint_create(ctypes.byref(self.c), rp, ctypes.byref(self.h)), "squint_create")
        self.n_params = int(self.lib.squint_param_count(ctypes.byref(self.c)))

    def _replay(self, ring):
        self._ring = ring     # keep the tensors alive
        obs = ring.get("obs")     # absent for state-based SAC (conv_layers = 0)
        return Replay(_ptr(obs), _ptr(ring["proprio"]), _ptr(ring["action"]), _ptr(ring["reward"]),
                      _ptr(ring["done"]), int(ring["proprio"].shape[0]))

    def set_replay(self, ring):
        _check(self.lib.squint_set_replay(self.h, ctypes.byref(self._replay(ring))), "squint_set_replay")

    def update(self, k=1, stats=True, stream=None, graph=True):
        st = (UpdateStats * k)() if stats else None
        fn = self.lib.squint_update if graph else self.lib.squint_update_eager
        _check(fn(self.h, int(k), st if stats else None, _stream(stream)), "squint_update")
        if not stats:
            return None
        return [{f: getattr(s, f) for f, _ in UpdateStats._fields_} for s in st]

    def update_async(self, k, stats=None, stream=None):
        """k updates as one graph without waiting; `stats` (a PinnedStats of at least k
        entries, or None) is filled by the stream."""
        if stats is not None and stats.k < k:
            raise ValueError("PinnedStats holds fewer than k entries")
        _check(self.lib.squint_update_async(self.h, int(k), ctypes.c_void_p(stats.ptr) if stats is not None else None,
                                            _stream(stream)), "squint_update_async")

    def update_check(self, stream=None):
        """Waits for the stream; raises if a bounded device wait of the updates ran out."""
        _check(self.lib.squint_update_check(self.h, _stream(stream)), "squint_update_check")

    def params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(self.lib.squint_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p), self.n_params),
               "squint_get_params")
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        _check(self.lib.squint_set_params(self.h, flat.ctypes.data_as(ctypes.c_void_p), flat.size),
               "squint_set_params")

    def state(self):
        n = ctypes.c_size_t(0)
        _check(self.lib.squint_get_state(self.h, None, ctypes.byref(n)), "squint_get_state")
        buf = (ctypes.c_uint8 * n.value)()
        _check(self.lib.squint_get_state(self.h, buf, ctypes.byref(n)), "squint_get_state")
        return bytes(buf)

    def set_state(self, blob):
        buf = (ctypes.c_uint8 * len(blob)).from_buffer_copy(blob)
        _check(self.lib.squint_set_state(self.h, buf, len(blob)), "squint_set_state")

    def debug(self, name, dtype=np.float32):
        n = ctypes.c_size_t(0)
        _check(self.lib.squint_debug_tensor(self.h, name.encode(), None, ctypes.byref(n)), "squint_debug_tensor")
        out = np.empty(n.value // np.dtype(dtype).itemsize, dtype=dtype)
        _check(self.lib.squint_debug_tensor(self.h, name.encode(), out.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.byref(n)), "squint_debug_tensor")
        return out

    def set_debug(self, name, value):
        _check(self.lib.squint_set_debug(self.h, name.encode(), int(value)), "squint_set_debug")

    def graph_kernel_count(self, k):
        return int(self.lib.squint_graph_kernel_count(self.h, int(k)))

    def device_bytes(self):
        """Device memory the learner allocated at creation (ring and inference buffers excluded)."""
        return int(self.lib.squint_device_bytes(self.h))

    def profile_update(self, stream=None):
        """One eager update timed per phase: {phase name: device ms}."""
        ms = (ctypes.c_float * 32)()
        n = ctypes.c_int(0)
        _check(self.lib.squint_profile_update(self.h, ms, 32, ctypes.byref(n), _stream(stream)),
               "squint_profile_update")
        return {self.lib.squint_phase_name(i).decode(): float(ms[i]) for i in range(n.value)}

    def profile_kernels(self, stream=None, cap=64):
        """One in-order eager update timed per launch: {class: (launches, ms, work, unit)}."""
        names = ctypes.create_string_buffer(32 * cap)
        launches = (ctypes.c_int * cap)()
        ms = (ctypes.c_float * cap)()
        work = (ctypes.c_double * cap)()
        unit = (ctypes.c_int * cap)()
        n = ctypes.c_int(0)
        _check(self.lib.squint_profile_kernels(self.h, cap, names, launches, ms, work, unit, ctypes.byref(n),
                                               _stream(stream)), "squint_profile_kernels")
        out = {}
        for i in range(min(n.value, cap)):
            nm = names.raw[32 * i:32 * (i + 1)].split(b"\0")[0].decode()
            out[nm] = (int(launches[i]), float(ms[i]), float(work[i]), "FLOP" if unit[i] == 0 else "B")
        return out

    def trace_update(self, stream=None, cap=512):
        """One update as the graph runs it, every launch timed: [(class, branch, start ms, end ms)]."""
        names = ctypes.create_string_buffer(32 * cap)
        lanes = (ctypes.c_int * cap)()
        t0 = (ctypes.c_float * cap)()
        t1 = (ctypes.c_float * cap)()
        n = ctypes.c_int(0)
        _check(self.lib.squint_trace_update(self.h, cap, names, lanes, t0, t1, ctypes.byref(n), _stream(stream)),
               "squint_trace_update")
        return [(names.raw[32 * i:32 * (i + 1)].split(b"\0")[0].decode(), int(lanes[i]), float(t0[i]), float(t1[i]))
                for i in range(min(n.value, cap))]

    def refresh_policy(self, stream=None):
        _check(self.lib.squint_refresh_policy(self.h, _stream(stream)), "squint_refresh_policy")

    @staticmethod
    def request(obs, proprio, actions, key, sample=True, group_id=0):
        """An ActRequest over caller-owned device tensors (obs uint8 [n,C,H,W], proprio f32 [n,P], actions f32 [n,A])."""
        return ActRequest(int(group_id), int(proprio.shape[0]), 0 if sample else 1, int(key), _ptr(obs),
                          _ptr(proprio), _ptr(actions))

    def act(self, requests, stream=None):
        arr = (ActRequest * len(requests))(*requests)
        _check(self.lib.squint_act(self.h, arr, len(requests), _stream(stream)), "squint_act")

    def serve_start(self, max_rows, mem_budget_bytes):
        _check(self.lib.squint_serve_start(self.h, int(max_rows), int(mem_budget_bytes)), "squint_serve_start")

    def serve_submit(self, req):
        t = ctypes.c_uint64(0)
        rc = self.lib.squint_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if rc == EAGAIN:
            return None
        _check(rc, "squint_serve_submit")
        return t.value

    def serve_poll(self, ticket, timeout_us=0):
        lat = ctypes.c_double(0)
        ver = ctypes.c_int64(0)
        rc = self.lib.squint_serve_poll(self.h, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(lat),
                                        ctypes.byref(ver))
        if rc == EAGAIN:
            return None
        _check(rc, "squint_serve_poll")
        return lat.value, ver.value

    def serve_poll_ex(self, ticket, timeout_us=0):
        """None if not done yet, else a dict: latency_us, policy_version, device_begin_us,
        device_end_us, slot, batch_rows."""
        r = ServeResult()
        rc = self.lib.squint_serve_poll_ex(self.h, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(r))
        if rc == EAGAIN:
            return None
        _check(rc, "squint_serve_poll_ex")
        return {f: getattr(r, f) for f, _ in ServeResult._fields_}

    def serve_info(self):
        a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int64(0)
        _check(self.lib.squint_serve_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "squint_serve_info")
        return {"slots": a.value, "slot_rows": b.value, "arena_bytes": c.value}

    def serve_stop(self):
        _check(self.lib.squint_serve_stop(self.h), "squint_serve_stop")

    def close(self):
        if self.h:
            self.lib.squint_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
