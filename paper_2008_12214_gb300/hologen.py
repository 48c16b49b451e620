"""ctypes binding of libhologen.so (include/hologen.h), argument marshalling only.

The functions carry the C names and take torch tensors (CUDA or CPU; CPU
tensors are host buffers the library copies through its own device
workspace) or None for optional outputs.  Every step of the computation runs
in the library's CUDA kernels; there is no other code path: if the library
is missing this module raises instead of computing anything.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhologen.so")

HG_SLM_BINARY, HG_SLM_LLEVEL, HG_SLM_AMPLITUDE = 0, 1, 2
HG_GS, HG_WGS, HG_OSPR, HG_ADOSPR, HG_LT, HG_DS, HG_SA = 0, 1, 2, 3, 4, 5, 6
NMET = 4

STATUS = {0: "HG_OK", 1: "HG_ERR_INVALID_ARG", 2: "HG_ERR_UNSUPPORTED_SIZE", 3: "HG_ERR_OOM",
          4: "HG_ERR_CUDA", 5: "HG_ERR_TIMEOUT", 6: "HG_ERR_NUMERIC", 7: "HG_ERR_TOO_LARGE"}
HG_NOALLOC_MAX_SIDE = 512


class HgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (where, STATUS.get(status, "?"), status))


class hg_opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("subframes", ctypes.c_int),
                ("precision", ctypes.c_int), ("use_graph", ctypes.c_int), ("pipeline", ctypes.c_int),
                ("autotune", ctypes.c_int), ("lt_start", ctypes.c_float), ("lt_grow", ctypes.c_int),
                ("modulated", ctypes.c_int), ("fresnel", ctypes.c_float), ("amp_clip", ctypes.c_float),
                ("sa_temp", ctypes.c_float), ("sa_cool", ctypes.c_float), ("host_chunks", ctypes.c_int)]


class hg_slm(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("levels", ctypes.c_int)]


_lib = None


def lib():
    """Load libhologen.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhologen.so is not built (run paper_2008_12214_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, I, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.hg_opts_size.argtypes = []
        L.hg_opts_size.restype = Z
        if L.hg_opts_size() != ctypes.sizeof(hg_opts):
            raise RuntimeError("libhologen.so was built with another hg_opts layout (%d bytes, binding %d): "
                               "rebuild it" % (L.hg_opts_size(), ctypes.sizeof(hg_opts)))
        L.hg_opts_default.argtypes = [ctypes.POINTER(hg_opts)]
        L.hg_opts_default.restype = None
        L.hg_supported_length.argtypes = [I]
        L.hg_supported_length.restype = I
        L.hg_plan_create.argtypes = [ctypes.POINTER(P), I, I, I, hg_slm, I, ctypes.POINTER(hg_opts)]
        L.hg_run.argtypes = [P, P, P, I, P, P]
        L.hg_get_metrics.argtypes = [P, P, Z]
        L.hg_replay.argtypes = [P, P, P]
        L.hg_get_phase.argtypes = [P, P]
        L.hg_set_illumination.argtypes = [P, P, P]
        L.hg_set_roi.argtypes = [P, P]
        L.hg_evaluate.argtypes = [P, P, P, P]
        L.hg_set_weights.argtypes = [P, P]
        L.hg_get_weights.argtypes = [P, P]
        L.hg_debug_step.argtypes = [P, P, P, P, P, P, P]
        L.hg_debug_loop_step.argtypes = [P, P, P, I, P, P, P, P]
        L.hg_sync.argtypes = [P]
        L.hg_last_launch_count.argtypes = [P]
        L.hg_last_launch_count.restype = I
        L.hg_pipelined.argtypes = [P]
        L.hg_pipelined.restype = I
        L.hg_plan_variant.argtypes = [P, I]
        L.hg_plan_variant.restype = ctypes.c_char_p
        L.hg_debug_inject.argtypes = [P, I, ctypes.c_uint64]
        L.hg_debug_inject.restype = I
        L.hg_profile_enable.argtypes = [P, I]
        L.hg_profile_enable.restype = I
        L.hg_profile_read.argtypes = [P, P]
        L.hg_profile_read.restype = I
        L.hg_plan_destroy.argtypes = [P]
        L.hg_plan_destroy.restype = None
        L.hg_group_create.argtypes = [ctypes.POINTER(P), I, P]
        L.hg_group_create.restype = I
        L.hg_group_run.argtypes = [P, P, P, I, P, P, P]
        L.hg_group_run.restype = I
        L.hg_group_sync.argtypes = [P, P]
        L.hg_group_sync.restype = I
        L.hg_group_launch_count.argtypes = [P]
        L.hg_group_launch_count.restype = I
        L.hg_group_set_schedule.argtypes = [P, I]
        L.hg_group_set_schedule.restype = I
        L.hg_group_destroy.argtypes = [P]
        L.hg_group_destroy.restype = None
        L.hg_run_noalloc.argtypes = [I, I, hg_slm, I, P, P, I, P, P, P]
        L.hg_run_noalloc.restype = I
        L.hg_cnn_create.argtypes = [ctypes.POINTER(P), I, I, I, ctypes.c_uint64, P]
        L.hg_cnn_destroy.argtypes = [P]
        L.hg_cnn_destroy.restype = None
        for name, args in (("hg_cnn_set_params", [P, P]), ("hg_cnn_get_params", [P, P]),
                           ("hg_cnn_get_grads", [P, P]), ("hg_cnn_forward", [P, P, I, P, P]),
                           ("hg_cnn_gradients", [P, P, P, I, P]),
                           ("hg_cnn_train_step", [P, P, P, I, ctypes.c_float, P]), ("hg_cnn_sync", [P]),
                           ("hg_cnn_apply_grads", [P, P, ctypes.c_float]),
                           ("hg_cnn_launch_count", [P]), ("hg_cnn_set_base_phase", [P, P]),
                           ("hg_conv3x3_forward", [P, I, I, I, I, P, I, P, I, P, P, P]),
                           ("hg_conv3x3_dgrad", [P, I, I, I, I, P, I, P, P, P]),
                           ("hg_conv3x3_wgrad", [P, P, I, I, I, I, I, P, P, P, Z, P]),
                           ("hg_conv_status", [P])):
            getattr(L, name).argtypes = args
            getattr(L, name).restype = I
        L.hg_cnn_create.restype = I
        L.hg_cnn_get_state.argtypes = [P, P, ctypes.POINTER(ctypes.c_int64)]
        L.hg_cnn_get_state.restype = I
        L.hg_cnn_set_state.argtypes = [P, P, ctypes.c_int64]
        L.hg_cnn_set_state.restype = I
        L.hg_conv3x3_wgrad_workspace.argtypes = [I, I, I, I, I]
        L.hg_conv3x3_wgrad_workspace.restype = Z
        L.hg_status_string.argtypes = [I]
        L.hg_status_string.restype = ctypes.c_char_p
        for name in ("hg_plan_create", "hg_run", "hg_get_metrics", "hg_replay", "hg_get_phase",
                     "hg_set_weights", "hg_get_weights", "hg_debug_step", "hg_debug_loop_step", "hg_sync",
                     "hg_set_illumination", "hg_set_roi", "hg_evaluate"):
            getattr(L, name).restype = I
        _lib = L
    return _lib


def _ck(st: int, where: str):
    if st != 0:
        raise HgError(st, where)


def _ptr(t, dtype=None, numel=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if numel is not None and t.numel() < numel:
        raise ValueError("%s holds %d elements, needs %d" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def hg_supported_length(n: int) -> bool:
    return bool(lib().hg_supported_length(int(n)))


def hg_status_string(st: int) -> str:
    return lib().hg_status_string(int(st)).decode()


def hg_plan_create(ny, nx, batch, slm_kind=HG_SLM_BINARY, levels=2, algo=HG_GS, stream=None,
                   seed=0, subframes=24, precision=0, use_graph=True, pipeline=-1, autotune=True,
                   lt_start=None, lt_grow=None, modulated=False, fresnel=0.0, amp_clip=None, sa_temp=None,
                   sa_cool=None, host_chunks=0):
    o = hg_opts()
    lib().hg_opts_default(ctypes.byref(o))
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream().cuda_stream
    o.stream = ctypes.c_void_p(int(stream or 0))
    o.seed = int(seed)
    o.subframes = int(subframes)
    o.precision = int(precision)
    o.use_graph = 1 if use_graph else 0
    o.pipeline = int(pipeline)
    o.autotune = int(autotune)
    if lt_start is not None:
        o.lt_start = float(lt_start)
    if lt_grow is not None:
        o.lt_grow = int(lt_grow)
    o.modulated = 1 if modulated else 0
    o.fresnel = float(fresnel)
    o.host_chunks = int(host_chunks)
    if amp_clip is not None:
        o.amp_clip = float(amp_clip)
    if sa_temp is not None:
        o.sa_temp = float(sa_temp)
    if sa_cool is not None:
        o.sa_cool = float(sa_cool)
    h = ctypes.c_void_p()
    _ck(lib().hg_plan_create(ctypes.byref(h), int(ny), int(nx), int(batch),
                             hg_slm(int(slm_kind), int(levels)), int(algo), ctypes.byref(o)),
        "hg_plan_create")
    return h


def hg_run(plan, target, init_phase, iters, holo_out=None, mse_out=None):
    _ck(lib().hg_run(plan, _ptr(target, torch.float32, name="target"),
                     _ptr(init_phase, torch.float32, name="init_phase"), int(iters),
                     _ptr(holo_out, torch.uint8, name="holo_out"),
                     _ptr(mse_out, torch.float64, name="mse_out")), "hg_run")


def hg_run_noalloc(ny, nx, target, init_phase, iters, holo_out=None, mse_out=None,
                   slm_kind=HG_SLM_BINARY, levels=2, algo=HG_GS, stream=None):
    """One GS/WGS run of one target in the library's fixed device region (no
    device allocation); CUDA tensors only.  Returns when the work is done."""
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream().cuda_stream
    _ck(lib().hg_run_noalloc(int(ny), int(nx), hg_slm(int(slm_kind), int(levels)), int(algo),
                             _ptr(target, torch.float32, ny * nx, name="target"),
                             _ptr(init_phase, torch.float32, ny * nx, name="init_phase"), int(iters),
                             _ptr(holo_out, torch.uint8, ny * nx, name="holo_out"),
                             _ptr(mse_out, torch.float64, iters, name="mse_out"),
                             ctypes.c_void_p(int(stream or 0))), "hg_run_noalloc")


def hg_get_metrics(plan, out):
    _ck(lib().hg_get_metrics(plan, _ptr(out, torch.float64, name="out"), out.numel()),
        "hg_get_metrics")


def hg_replay(plan, holo, intensity_out):
    _ck(lib().hg_replay(plan, _ptr(holo, torch.uint8, name="holo"),
                        _ptr(intensity_out, torch.float32, name="intensity_out")), "hg_replay")


def hg_get_phase(plan, phase_out):
    _ck(lib().hg_get_phase(plan, _ptr(phase_out, torch.float32, name="phase_out")), "hg_get_phase")


def hg_set_illumination(plan, amp=None, phase=None):
    _ck(lib().hg_set_illumination(plan, _ptr(amp, torch.float32, name="amp"),
                                  _ptr(phase, torch.float32, name="phase")), "hg_set_illumination")


def hg_set_roi(plan, roi=None):
    _ck(lib().hg_set_roi(plan, _ptr(roi, torch.uint8, name="roi")), "hg_set_roi")


def hg_evaluate(plan, holo, target, out):
    _ck(lib().hg_evaluate(plan, _ptr(holo, torch.uint8, name="holo"), _ptr(target, torch.float32, name="target"),
                          _ptr(out, torch.float64, name="out")), "hg_evaluate")


def hg_set_weights(plan, w):
    _ck(lib().hg_set_weights(plan, _ptr(w, torch.float32, name="w")), "hg_set_weights")


def hg_get_weights(plan, w_out):
    _ck(lib().hg_get_weights(plan, _ptr(w_out, torch.float32, name="w_out")), "hg_get_weights")


def hg_debug_step(plan, target, phase_in, h_out=None, holo_out=None, replay_out=None,
                  metrics_out=None):
    _ck(lib().hg_debug_step(plan, _ptr(target, torch.float32, name="target"),
                            _ptr(phase_in, torch.float32, name="phase_in"),
                            _ptr(h_out, torch.complex64, name="h_out"),
                            _ptr(holo_out, torch.uint8, name="holo_out"),
                            _ptr(replay_out, torch.complex64, name="replay_out"),
                            _ptr(metrics_out, torch.float64, name="metrics_out")), "hg_debug_step")


def hg_debug_loop_step(plan, target, holo_in, k=0, row_out=None, holo_out=None, col_out=None,
                       metrics_out=None):
    _ck(lib().hg_debug_loop_step(plan, _ptr(target, torch.float32, name="target"),
                                 _ptr(holo_in, torch.uint8, name="holo_in"), int(k),
                                 _ptr(row_out, torch.complex64, name="row_out"),
                                 _ptr(holo_out, torch.uint8, name="holo_out"),
                                 _ptr(col_out, torch.complex64, name="col_out"),
                                 _ptr(metrics_out, torch.float64, name="metrics_out")), "hg_debug_loop_step")


def hg_sync(plan):
    _ck(lib().hg_sync(plan), "hg_sync")


def hg_last_launch_count(plan) -> int:
    return lib().hg_last_launch_count(plan)


def hg_pipelined(plan) -> int:
    return lib().hg_pipelined(plan)


def hg_plan_variant(plan, which) -> str:
    return lib().hg_plan_variant(plan, int(which)).decode()


def hg_debug_inject(plan, drop_job, wait_ns):
    _ck(lib().hg_debug_inject(plan, int(drop_job), int(wait_ns)), "hg_debug_inject")


def hg_profile_enable(plan, max_passes):
    _ck(lib().hg_profile_enable(plan, int(max_passes)), "hg_profile_enable")


def hg_profile_read(plan):
    """{row ms, row passes, column ms, column passes} since the last read."""
    out = (ctypes.c_double * 4)()
    _ck(lib().hg_profile_read(plan, ctypes.cast(out, ctypes.c_void_p)), "hg_profile_read")
    return list(out)


def hg_plan_destroy(plan):
    if plan:
        lib().hg_plan_destroy(plan)


def _ptr_array(ts, dtype, name):
    if ts is None:
        return None
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        p = _ptr(t, dtype, name=name)
        arr[i] = p.value if p is not None else None
    return ctypes.cast(arr, ctypes.c_void_p), arr


def hg_group_create(plans):
    """plans: list of Plan objects or raw handles."""
    hs = [p.h if isinstance(p, Plan) else p for p in plans]
    arr = (ctypes.c_void_p * len(hs))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in hs])
    g = ctypes.c_void_p()
    _ck(lib().hg_group_create(ctypes.byref(g), len(hs), ctypes.cast(arr, ctypes.c_void_p)), "hg_group_create")
    return g


def hg_group_run(group, targets, init_phases, iters, holo_out=None, mse_out=None, stream=None):
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream().cuda_stream
    keep = []
    args = []
    for ts, dt, nm in ((targets, torch.float32, "targets"), (init_phases, torch.float32, "init_phases"),
                       (holo_out, torch.uint8, "holo_out"), (mse_out, torch.float64, "mse_out")):
        r = _ptr_array(ts, dt, nm)
        keep.append(r)
        args.append(None if r is None else r[0])
    _ck(lib().hg_group_run(group, args[0], args[1], int(iters), args[2], args[3],
                           ctypes.c_void_p(int(stream or 0))), "hg_group_run")


def hg_group_sync(group, stream=None):
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream().cuda_stream
    _ck(lib().hg_group_sync(group, ctypes.c_void_p(int(stream or 0))), "hg_group_sync")


def hg_group_launch_count(group) -> int:
    return lib().hg_group_launch_count(group)


HG_GROUP_SERIAL, HG_GROUP_CONCURRENT = 0, 1


def hg_group_set_schedule(group, schedule):
    _ck(lib().hg_group_set_schedule(group, int(schedule)), "hg_group_set_schedule")


def hg_group_destroy(group):
    if group:
        lib().hg_group_destroy(group)


class Plan:
    """Owning wrapper of an hg_plan with shapes attached (same calls, same
    semantics as the C functions)."""

    def __init__(self, ny, nx, batch=1, slm_kind=HG_SLM_BINARY, levels=2, algo=HG_GS, **kw):
        self.ny, self.nx, self.batch = int(ny), int(nx), int(batch)
        self.algo = algo
        self.subframes = int(kw.get("subframes", 24)) if algo == HG_OSPR else 1
        self.h = hg_plan_create(ny, nx, batch, slm_kind, levels, algo, **kw)
        self.iters = 0

    def close(self):
        if self.h:
            hg_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, target, init_phase=None, iters=1, holo_out=None, mse_out=None):
        hg_run(self.h, target, init_phase, iters, holo_out, mse_out)
        self.iters = 1 if self.algo == HG_OSPR else int(iters)

    def metrics(self, device="cuda"):
        out = torch.empty((self.batch, self.iters, NMET), dtype=torch.float64, device=device)
        hg_get_metrics(self.h, out)
        return out

    def sync(self):
        hg_sync(self.h)

    def set_illumination(self, amp=None, phase=None):
        hg_set_illumination(self.h, amp, phase)

    def set_roi(self, roi=None):
        hg_set_roi(self.h, roi)

    def evaluate(self, holo, target, device="cuda"):
        """[batch][5] {intensity MSE, amplitude MSE, efficiency, SSIM, sum |R|^2}."""
        out = torch.empty((self.batch, 5), dtype=torch.float64, device=device)
        hg_evaluate(self.h, holo, target, out)
        return out


# ------------------------------------------------------------------ warm start

HG_CNN_NPARAMS = 1946338


def _stream(stream):
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream().cuda_stream
    return ctypes.c_void_p(int(stream or 0))


def hg_cnn_create(height, width, max_batch, seed=0, stream=None):
    h = ctypes.c_void_p()
    _ck(lib().hg_cnn_create(ctypes.byref(h), int(height), int(width), int(max_batch), int(seed), _stream(stream)),
        "hg_cnn_create")
    return h


def hg_cnn_destroy(net):
    lib().hg_cnn_destroy(net)


def hg_cnn_set_params(net, params):
    _ck(lib().hg_cnn_set_params(net, _ptr(params, torch.float32, HG_CNN_NPARAMS, "params")), "hg_cnn_set_params")


def hg_cnn_get_params(net, params):
    _ck(lib().hg_cnn_get_params(net, _ptr(params, torch.float32, HG_CNN_NPARAMS, "params")), "hg_cnn_get_params")


def hg_cnn_get_state(net, state) -> int:
    """Fills state (3 x HG_CNN_NPARAMS floats) and returns Adam's step count."""
    st = ctypes.c_int64()
    _ck(lib().hg_cnn_get_state(net, _ptr(state, torch.float32, 3 * HG_CNN_NPARAMS, "state"), ctypes.byref(st)),
        "hg_cnn_get_state")
    return st.value


def hg_cnn_set_state(net, state, step):
    _ck(lib().hg_cnn_set_state(net, _ptr(state, torch.float32, 3 * HG_CNN_NPARAMS, "state"), int(step)),
        "hg_cnn_set_state")


def hg_cnn_get_grads(net, grads):
    _ck(lib().hg_cnn_get_grads(net, _ptr(grads, torch.float32, HG_CNN_NPARAMS, "grads")), "hg_cnn_get_grads")


def hg_cnn_forward(net, target, batch, cs_out=None, phase_out=None):
    _ck(lib().hg_cnn_forward(net, _ptr(target, torch.float32, name="target"), int(batch),
                             _ptr(cs_out, torch.float32, name="cs_out"),
                             _ptr(phase_out, torch.float32, name="phase_out")), "hg_cnn_forward")


def hg_cnn_gradients(net, target, phase_label, batch, loss_out=None):
    _ck(lib().hg_cnn_gradients(net, _ptr(target, torch.float32, name="target"),
                               _ptr(phase_label, torch.float32, name="phase_label"), int(batch),
                               _ptr(loss_out, torch.float64, name="loss_out")), "hg_cnn_gradients")


def hg_cnn_train_step(net, target, phase_label, batch, lr, loss_out=None):
    _ck(lib().hg_cnn_train_step(net, _ptr(target, torch.float32, name="target"),
                                _ptr(phase_label, torch.float32, name="phase_label"), int(batch), float(lr),
                                _ptr(loss_out, torch.float64, name="loss_out")), "hg_cnn_train_step")


def hg_cnn_apply_grads(net, grads, lr):
    _ck(lib().hg_cnn_apply_grads(net, _ptr(grads, torch.float32, HG_CNN_NPARAMS, name="grads"), float(lr)),
        "hg_cnn_apply_grads")


def hg_cnn_set_base_phase(net, base):
    """base: float32 [H][W] radians (device or host tensor) or None to remove it."""
    _ck(lib().hg_cnn_set_base_phase(net, _ptr(base, torch.float32, name="base")), "hg_cnn_set_base_phase")


def hg_cnn_sync(net):
    _ck(lib().hg_cnn_sync(net), "hg_cnn_sync")


def hg_cnn_launch_count(net) -> int:
    return lib().hg_cnn_launch_count(net)


def hg_conv3x3_forward(x, B, H, W, Cin, w, Cout, bias, relu, mask, y, stream=None):
    _ck(lib().hg_conv3x3_forward(_ptr(x, torch.bfloat16, name="x"), B, H, W, Cin, _ptr(w, torch.bfloat16, name="w"),
                                 Cout, _ptr(bias, torch.float32, name="bias"), int(relu),
                                 _ptr(mask, torch.bfloat16, name="mask"), _ptr(y, torch.bfloat16, name="y"),
                                 _stream(stream)), "hg_conv3x3_forward")


def hg_conv3x3_dgrad(dy, B, H, W, Cout, w_rot, Cin, mask, dx, stream=None):
    _ck(lib().hg_conv3x3_dgrad(_ptr(dy, torch.bfloat16, name="dy"), B, H, W, Cout,
                               _ptr(w_rot, torch.bfloat16, name="w_rot"), Cin, _ptr(mask, torch.bfloat16, name="mask"),
                               _ptr(dx, torch.bfloat16, name="dx"), _stream(stream)), "hg_conv3x3_dgrad")


def hg_conv3x3_wgrad_workspace(B, H, W, Cin, Cout) -> int:
    return int(lib().hg_conv3x3_wgrad_workspace(B, H, W, Cin, Cout))


def hg_conv3x3_wgrad(x, dy, B, H, W, Cin, Cout, dw, db, workspace, stream=None):
    _ck(lib().hg_conv3x3_wgrad(_ptr(x, torch.bfloat16, name="x"), _ptr(dy, torch.bfloat16, name="dy"), B, H, W, Cin,
                               Cout, _ptr(dw, torch.float32, name="dw"), _ptr(db, torch.float32, name="db"),
                               _ptr(workspace, torch.uint8, name="workspace"), workspace.numel(), _stream(stream)),
        "hg_conv3x3_wgrad")


def hg_conv_status(stream=None):
    _ck(lib().hg_conv_status(_stream(stream)), "hg_conv_status")


class CNN:
    """Owning wrapper of an hg_cnn handle."""

    def __init__(self, height, width, max_batch, seed=0, stream=None):
        self.h = hg_cnn_create(height, width, max_batch, seed, stream)
        self.height, self.width, self.max_batch = height, width, max_batch

    def close(self):
        if self.h is not None and self.h.value:
            hg_cnn_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
