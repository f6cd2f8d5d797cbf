"""ctypes binding of libj2d5pt.so (include/j2d5pt.h) -- argument marshalling only.

Every computation runs in the library's CUDA kernels.  The module fails
loudly when the library is missing; there is no fallback.  torch is used for
device memory and streams.

Functions keep the C names (``j2d5pt_plan``, ``j2d5pt_run``, ...).  ``Plan``
wraps a plan handle with helpers that allocate device buffers in the plan's
layout and move dense (ny+2, nx+2) arrays (ring included) in and out.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libj2d5pt.so")
# the same library built with every memory access of the blocked kernels
# tested against its buffer (J2D_BOUNDS_CHECK): for tests, not for speed
LIB_CHECKED_PATH = os.path.join(_HERE, "libj2d5pt_checked.so")

J2D_F64, J2D_F32 = 0, 1
J2D_OK, J2D_ERR_ARG, J2D_ERR_ALIGN, J2D_ERR_NOMEM, J2D_ERR_DEVICE = 0, 1, 2, 3, 4
J2D_ERR_UNSUPPORTED, J2D_ERR_TIMEOUT, J2D_ERR_BOUNDS = 5, 6, 7
ALGO = {"auto": 0, "onestep": 1, "resident": 2, "bands": 3, "tiles": 4, "skewed": 5, "stream": 6}
OPT = {"algo": 0, "depth": 1, "tile_wx": 2, "ctas": 3, "timeout_ms": 4, "verbose": 5, "graph": 6, "timing": 7, "fault_inject": 8,
       "int_path": 9, "sweep_steps": 10}
STATUS_NAMES = {0: "J2D_OK", 1: "J2D_ERR_ARG", 2: "J2D_ERR_ALIGN", 3: "J2D_ERR_NOMEM", 4: "J2D_ERR_DEVICE",
                5: "J2D_ERR_UNSUPPORTED", 6: "J2D_ERR_TIMEOUT", 7: "J2D_ERR_BOUNDS"}

_lib = None
_lib_checked = None


class J2DError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


def load():
    """Load libj2d5pt.so (built by paper_2306_03336_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        _lib = _open(LIB_PATH)
    return _lib


def load_checked():
    """Load the bounds-checked build libj2d5pt_checked.so (a separate handle
    with the same functions); raise if absent."""
    global _lib_checked
    if _lib_checked is None:
        _lib_checked = _open(LIB_CHECKED_PATH)
    return _lib_checked


def _open(path):
    if not os.path.exists(path):
        raise RuntimeError("%s is not built (run __graft_entry__.build()); "
                           "the CUDA library is required, there is no fallback" % os.path.basename(path))
    lib = ctypes.CDLL(path)
    P, I, L, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "j2d5pt_plan": [PP, I, I, I, P],
        "j2d5pt_plan_batched": [PP, I, P, P, I, P],
        "j2d9pt_plan": [PP, I, I, I, P],
        "j2d9pt_measure_exact_rate": [ctypes.POINTER(D)],
        "j2d5pt_plan_destroy": [P],
        "j2d5pt_layout": [P, I, ctypes.POINTER(L), ctypes.POINTER(L)],
        "j2d5pt_set_weights": [P, I, P],
        "j2d5pt_set_option": [P, I, L],
        "j2d5pt_get_option": [P, I, ctypes.POINTER(L)],
        "j2d5pt_describe": [P, ctypes.c_char_p, ctypes.c_size_t],
        "j2d5pt_run": [P, P, P, L, P],
        "j2d5pt_run_batched": [P, P, P, L, P],
        "j2d5pt_run_host": [P, P, P, L],
        "j2d5pt_run_states": [P, P, P, L, P],
        "j2d5pt_run_adjoint": [P, P, P, L, P],
        "j2d5pt_weight_grad": [P, P, P, P, P],
        "j2d5pt_adjoint_step_wgrad": [P, P, P, P, P, P],
        "j2d5pt_sync_status": [P],
        "j2d5pt_autotune": [P, P, P, L, P],
        "j2d5pt_autotune_batched": [P, P, P, L, P],
        "j2d5pt_measure_fma_rate": [I, ctypes.POINTER(D)],
        "j2d5pt_weight_grad_noalloc": [I, I, I, P, P, P, P],
        "j2d5pt_kernel_time": [P, ctypes.POINTER(D)],
        "j2d5pt_measure_exact_rate": [ctypes.POINTER(D)],
        "j2d5pt_measure_smem_bandwidth": [ctypes.POINTER(D)],
        "j2d5pt_arith_info": [ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(I)],
        "j2d5pt_stream_geometry": [I, I, I, I, I, L, ctypes.POINTER(L)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.j2d5pt_last_error.argtypes = []
    lib.j2d5pt_last_error.restype = ctypes.c_char_p
    lib.j2d5pt_kernel_launches.argtypes = []
    lib.j2d5pt_kernel_launches.restype = ctypes.c_long
    lib.j2d5pt_version.argtypes = []
    lib.j2d5pt_version.restype = ctypes.c_char_p
    return lib


def _check(status):
    if status != J2D_OK:
        raise J2DError(status, load().j2d5pt_last_error().decode())


def j2d5pt_last_error():
    return load().j2d5pt_last_error().decode()


def j2d5pt_kernel_launches():
    return int(load().j2d5pt_kernel_launches())


def j2d5pt_version():
    return load().j2d5pt_version().decode()


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr() if hasattr(t, "data_ptr") else int(t))


def j2d5pt_plan(nx, ny, dtype, weights):
    h = ctypes.c_void_p()
    w = np.ascontiguousarray(weights, dtype=np.float64)
    _check(load().j2d5pt_plan(ctypes.byref(h), int(nx), int(ny), int(dtype), w.ctypes.data_as(ctypes.c_void_p)))
    return h


def j2d9pt_plan(nx, ny, dtype, weights):
    """Plan for the 3x3 box stencil: nine weights, rows y-1, y, y+1, columns x-1, x, x+1."""
    h = ctypes.c_void_p()
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
    if w.size != 9:
        raise ValueError("the box stencil takes nine weights")
    _check(load().j2d9pt_plan(ctypes.byref(h), int(nx), int(ny), int(dtype), w.ctypes.data_as(ctypes.c_void_p)))
    return h


def j2d9pt_measure_exact_rate():
    r = ctypes.c_double()
    _check(load().j2d9pt_measure_exact_rate(ctypes.byref(r)))
    return r.value


def j2d5pt_plan_batched(nx, ny, dtype, weights):
    h = ctypes.c_void_p()
    a = np.ascontiguousarray(nx, dtype=np.int32)
    b = np.ascontiguousarray(ny, dtype=np.int32)
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
    _check(load().j2d5pt_plan_batched(ctypes.byref(h), len(a), a.ctypes.data_as(ctypes.c_void_p),
                                      b.ctypes.data_as(ctypes.c_void_p), int(dtype),
                                      w.ctypes.data_as(ctypes.c_void_p)))
    return h


def j2d5pt_plan_destroy(h):
    _check(load().j2d5pt_plan_destroy(h))


def j2d5pt_set_weights(h, index, weights):
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(5)
    _check(load().j2d5pt_set_weights(h, int(index), w.ctypes.data_as(ctypes.c_void_p)))


def j2d5pt_layout(h, index=0):
    p, o = ctypes.c_long(), ctypes.c_long()
    _check(load().j2d5pt_layout(h, int(index), ctypes.byref(p), ctypes.byref(o)))
    return p.value, o.value


def j2d5pt_set_option(h, opt, value):
    _check(load().j2d5pt_set_option(h, OPT[opt] if isinstance(opt, str) else int(opt), int(value)))


def j2d5pt_get_option(h, opt):
    v = ctypes.c_long()
    _check(load().j2d5pt_get_option(h, OPT[opt] if isinstance(opt, str) else int(opt), ctypes.byref(v)))
    return v.value


def j2d5pt_describe(h):
    buf = ctypes.create_string_buffer(512)
    _check(load().j2d5pt_describe(h, buf, 512))
    return buf.value.decode()


def j2d5pt_run(h, src, dst, steps, stream=None):
    _check(load().j2d5pt_run(h, _ptr(src), _ptr(dst), int(steps), _stream_ptr(stream)))


def j2d5pt_run_batched(h, srcs, dsts, steps, stream=None):
    n = len(srcs)
    a = (ctypes.c_void_p * n)(*[_ptr(t).value for t in srcs])
    b = (ctypes.c_void_p * n)(*[_ptr(t).value for t in dsts])
    _check(load().j2d5pt_run_batched(h, ctypes.cast(a, ctypes.c_void_p), ctypes.cast(b, ctypes.c_void_p),
                                     int(steps), _stream_ptr(stream)))


def j2d5pt_run_host(h, h_in, h_out, steps):
    _check(load().j2d5pt_run_host(h, h_in.ctypes.data_as(ctypes.c_void_p), h_out.ctypes.data_as(ctypes.c_void_p),
                                  int(steps)))


def j2d5pt_run_states(h, src, states, steps, stream=None):
    _check(load().j2d5pt_run_states(h, _ptr(src), _ptr(states), int(steps), _stream_ptr(stream)))


def j2d5pt_run_adjoint(h, lam_T, lam_0, steps, stream=None):
    _check(load().j2d5pt_run_adjoint(h, _ptr(lam_T), _ptr(lam_0), int(steps), _stream_ptr(stream)))


def j2d5pt_weight_grad(h, u_t, lam_t1, dw, stream=None):
    _check(load().j2d5pt_weight_grad(h, _ptr(u_t), _ptr(lam_t1), _ptr(dw), _stream_ptr(stream)))


def j2d5pt_adjoint_step_wgrad(h, u_t, lam_t1, lam_t, dw, stream=None):
    _check(load().j2d5pt_adjoint_step_wgrad(h, _ptr(u_t), _ptr(lam_t1), _ptr(lam_t), _ptr(dw), _stream_ptr(stream)))


def j2d5pt_weight_grad_noalloc(nx, ny, dtype, u_t, lam_t1, dw, stream=None):
    _check(load().j2d5pt_weight_grad_noalloc(int(nx), int(ny), int(dtype), _ptr(u_t), _ptr(lam_t1), _ptr(dw),
                                             _stream_ptr(stream)))


def j2d5pt_sync_status(h):
    _check(load().j2d5pt_sync_status(h))


def j2d5pt_autotune(h, src, dst, steps, stream=None):
    _check(load().j2d5pt_autotune(h, _ptr(src), _ptr(dst), int(steps), _stream_ptr(stream)))


def j2d5pt_autotune_batched(h, srcs, dsts, steps, stream=None):
    n = len(srcs)
    a = (ctypes.c_void_p * n)(*[_ptr(t).value for t in srcs])
    b = (ctypes.c_void_p * n)(*[_ptr(t).value for t in dsts])
    _check(load().j2d5pt_autotune_batched(h, ctypes.cast(a, ctypes.c_void_p), ctypes.cast(b, ctypes.c_void_p),
                                          int(steps), _stream_ptr(stream)))


def j2d5pt_kernel_time(h):
    ms = ctypes.c_double()
    _check(load().j2d5pt_kernel_time(h, ctypes.byref(ms)))
    return ms.value


def j2d5pt_measure_fma_rate(dtype):
    r = ctypes.c_double()
    _check(load().j2d5pt_measure_fma_rate(int(dtype), ctypes.byref(r)))
    return r.value


def j2d5pt_measure_smem_bandwidth():
    r = ctypes.c_double()
    _check(load().j2d5pt_measure_smem_bandwidth(ctypes.byref(r)))
    return r.value


def j2d5pt_measure_exact_rate():
    r = ctypes.c_double()
    _check(load().j2d5pt_measure_exact_rate(ctypes.byref(r)))
    return r.value


def j2d5pt_arith_info():
    """(exact_mask, exact_guard): which FP64 cells take the integer path."""
    m, g = ctypes.c_uint(), ctypes.c_int()
    _check(load().j2d5pt_arith_info(ctypes.byref(m), ctypes.byref(g)))
    return int(m.value), int(g.value)


def j2d5pt_stream_geometry(nx, ny, dtype, depth, resident_warps, shape=5):
    """The stream schedule's geometry (host arithmetic): a dict with the steps
    per pass, halo columns G, stored columns per band, bands, rows per run H
    and runs per band."""
    out = (ctypes.c_long * 6)()
    _check(load().j2d5pt_stream_geometry(int(nx), int(ny), _DT[dtype], int(shape), int(depth), int(resident_warps),
                                         out))
    return dict(zip(("depth", "G", "vw", "bands", "H", "runs"), (int(v) for v in out)))


_DT = {"f64": J2D_F64, "f32": J2D_F32, np.float64: J2D_F64, np.float32: J2D_F32}


class Plan:
    """A plan handle plus layout helpers.  ``dtype`` is "f64" or "f32"."""

    def __init__(self, nx, ny=None, dtype="f64", weights=None, batched=False):
        self.dtype = dtype
        self.code = _DT[dtype]
        self.box = not batched and np.asarray(weights).size == 9
        if self.box:
            self.sizes = [(int(nx), int(ny))]
            self.weights = np.asarray(weights, dtype=np.float64).reshape(1, 9)
            self.handle = j2d9pt_plan(nx, ny, self.code, self.weights[0])
        elif batched:
            sizes = list(nx)
            self.sizes = [(int(a), int(b)) for a, b in sizes]
            w = np.asarray(weights, dtype=np.float64).reshape(len(sizes), 5)
            self.handle = j2d5pt_plan_batched([s[0] for s in sizes], [s[1] for s in sizes], self.code, w)
            self.weights = w
        else:
            self.sizes = [(int(nx), int(ny))]
            self.weights = np.asarray(weights, dtype=np.float64).reshape(1, 5)
            self.handle = j2d5pt_plan(nx, ny, self.code, self.weights[0])
        self.batched = batched
        self.layouts = [j2d5pt_layout(self.handle, i) for i in range(len(self.sizes))]

    @classmethod
    def batch(cls, sizes, dtype, weights):
        return cls(sizes, None, dtype, weights, batched=True)

    @classmethod
    def box9(cls, nx, ny, dtype, weights):
        """A 3x3 box (j2d9pt) plan; weights row by row from the y-1 row, x-1 first."""
        w = np.asarray(weights, dtype=np.float64).reshape(-1)
        if w.size != 9:
            raise ValueError("the box stencil takes nine weights")
        return cls(nx, ny, dtype, w)

    def close(self):
        if self.handle is not None:
            j2d5pt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.dtype == "f64" else torch.float32

    @property
    def np_dtype(self):
        return np.float64 if self.dtype == "f64" else np.float32

    def empty(self, i=0):
        """Zeroed device buffer in grid i's layout, shape (ny+2, pitch)."""
        import torch
        nx, ny = self.sizes[i]
        pitch, _ = self.layouts[i]
        return torch.zeros((ny + 2, pitch), dtype=self.torch_dtype, device="cuda")

    def view(self, t, i=0):
        """The logical (ny+2, nx+2) window of a buffer in plan layout."""
        nx, _ = self.sizes[i]
        _, off = self.layouts[i]
        return t[:, off:off + nx + 2]

    def to_device(self, a, i=0):
        import torch
        t = self.empty(i)
        self.view(t, i).copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=self.np_dtype)))
        return t

    def to_host(self, t, i=0):
        return self.view(t, i).cpu().numpy().astype(np.float64)

    def set(self, opt, value):
        j2d5pt_set_option(self.handle, opt, ALGO[value] if opt == "algo" and isinstance(value, str) else value)
        return self

    def get(self, opt):
        return j2d5pt_get_option(self.handle, opt)

    def kernel_time(self):
        return j2d5pt_kernel_time(self.handle)

    def set_weights(self, weights, i=0):
        j2d5pt_set_weights(self.handle, i, weights)
        self.weights[i] = np.asarray(weights, dtype=np.float64).reshape(5)
        return self

    def describe(self):
        return j2d5pt_describe(self.handle)

    def run(self, src, dst, steps, stream=None):
        j2d5pt_run(self.handle, src, dst, steps, stream)
        return dst

    def run_batched(self, srcs, dsts, steps, stream=None):
        j2d5pt_run_batched(self.handle, srcs, dsts, steps, stream)
        return dsts

    def run_adjoint(self, lam_T, lam_0, steps, stream=None):
        j2d5pt_run_adjoint(self.handle, lam_T, lam_0, steps, stream)
        return lam_0

    def weight_grad(self, u_t, lam_t1, dw, stream=None):
        j2d5pt_weight_grad(self.handle, u_t, lam_t1, dw, stream)
        return dw

    def adjoint_step_wgrad(self, u_t, lam_t1, lam_t, dw, stream=None):
        """lam_t = one adjoint step of lam_t1; dw += weight gradient of (u_t, lam_t1)."""
        j2d5pt_adjoint_step_wgrad(self.handle, u_t, lam_t1, lam_t, dw, stream)
        return lam_t

    def empty_states(self, steps):
        """Zeroed device buffer for `steps` states of grid 0, shape (steps, ny+2, pitch)."""
        import torch
        nx, ny = self.sizes[0]
        pitch, _ = self.layouts[0]
        return torch.zeros((steps, ny + 2, pitch), dtype=self.torch_dtype, device="cuda")

    def run_states(self, src, states, steps, stream=None):
        """Every state of a forward run: states[t-1] <- state t, t = 1..steps
        (states from empty_states or a same-shaped slice of one)."""
        j2d5pt_run_states(self.handle, src, states, steps, stream)
        return states

    def run_host(self, a, steps, out=None):
        """End to end on host arrays: dense (ny+2, nx+2) in, same shape out
        (`out`, if given, e.g. pinned memory for full copy bandwidth)."""
        a = np.ascontiguousarray(a, dtype=self.np_dtype)
        if out is None:
            out = np.empty_like(a)
        elif out.shape != a.shape or out.dtype != a.dtype or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a contiguous array like the input")
        j2d5pt_run_host(self.handle, a, out, steps)
        return out

    def sync(self):
        j2d5pt_sync_status(self.handle)

    def autotune(self, src, dst, steps, stream=None):
        j2d5pt_autotune(self.handle, src, dst, steps, stream)
        return self.describe()

    def autotune_batched(self, srcs, dsts, steps, stream=None):
        j2d5pt_autotune_batched(self.handle, srcs, dsts, steps, stream)
        return self.describe()
