"""ctypes binding of libxslam (include/xslam.h): argument marshalling only.

Every computation runs in the CUDA kernels behind the C ABI; this module converts torch tensors and
numpy arrays to pointers, checks shapes, and turns status codes into exceptions. It fails loudly
if the shared library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

POSE0, POSE, TRUNC, DEPTH, POSE_TRACKED = 0, 1, 2, 3, 4
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTRACK, ESTATE = range(7)
PIPELINE = 4  # XSLAM_PIPELINE: frames submitted and not yet waited for
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTRACK", 6: "ESTATE"}
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libxslam.so")

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_float_p = ctypes.POINTER(ctypes.c_float)
_c_int_p = ctypes.POINTER(ctypes.c_int)


class Seed(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("index", ctypes.c_int), ("h", ctypes.c_double)]


class Intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int), ("height", ctypes.c_int)]


class Config(ctypes.Structure):
    _fields_ = [("icp_levels", ctypes.c_int), ("icp_iters", ctypes.c_int * 4),
                ("dist_gate_m", ctypes.c_float), ("normal_gate_deg", ctypes.c_float),
                ("disc_gate_m", ctypes.c_float), ("min_corr_frac", ctypes.c_float),
                ("ray_step_vox", ctypes.c_float), ("depth_min_m", ctypes.c_float),
                ("depth_max_m", ctypes.c_float), ("pyr_range_m", ctypes.c_float),
                ("bilateral", ctypes.c_int), ("w_max", ctypes.c_float), ("icp_newton", ctypes.c_int),
                ("icp_newton_eta", ctypes.c_float), ("icp_seed", ctypes.c_int), ("icp_stop", ctypes.c_float)]


class XSlamError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"xslam {_STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None

# (name, restype, argtypes): every symbol declared in include/xslam.h
SYMBOLS = [
    ("xslam_default_config", None, [ctypes.POINTER(Config)]),
    ("xslam_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_float, ctypes.c_float, _c_float_p, ctypes.POINTER(Intrinsics),
                                    ctypes.POINTER(Config), ctypes.c_int, ctypes.c_void_p]),
    ("xslam_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("xslam_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("xslam_set_pose", ctypes.c_int, [ctypes.c_void_p, _c_double_p]),
    ("xslam_frame", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Seed), ctypes.c_int,
                                   _c_double_p, _c_double_p, _c_double_p]),
    ("xslam_sync", ctypes.c_int, [ctypes.c_void_p, _c_int_p]),
    ("xslam_frame_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Seed),
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]),
    ("xslam_frame_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, _c_double_p, _c_double_p, _c_double_p]),
    ("xslam_raycast", ctypes.c_int, [ctypes.c_void_p, _c_double_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("xslam_grad", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _c_double_p, ctypes.c_int, _c_double_p,
                                  _c_double_p, _c_double_p]),
    ("xslam_grad_plain64", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _c_double_p, _c_double_p, _c_double_p,
                                          _c_double_p]),
    ("xslam_grad_tsdf", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _c_double_p, ctypes.c_int, _c_double_p,
                                       _c_double_p, _c_double_p, ctypes.POINTER(ctypes.c_longlong)]),
    ("xslam_grad_tsdf_plain64", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _c_double_p, _c_double_p,
                                               _c_double_p, _c_double_p, ctypes.POINTER(ctypes.c_longlong)]),
    ("xslam_read_tsdf", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("xslam_set_lanes", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Seed), ctypes.c_int]),
    ("xslam_set_pose_lanes", ctypes.c_int, [ctypes.c_void_p, _c_double_p]),
    ("xslam_get_pose_lanes", ctypes.c_int, [ctypes.c_void_p, _c_double_p]),
    ("xslam_write_tsdf", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("xslam_measure", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("xslam_integrate", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("xslam_set_model", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       _c_double_p]),
    ("xslam_icp_system", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_double_p, _c_double_p, _c_int_p]),
    ("xslam_profile", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("xslam_profile_read", ctypes.c_int, [ctypes.c_void_p, _c_double_p, ctypes.POINTER(ctypes.c_longlong),
                                          _c_double_p]),
    ("xslam_icp_system_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Intrinsics),
                                                ctypes.c_void_p, _c_double_p, _c_double_p, ctypes.POINTER(Seed),
                                                ctypes.c_int, ctypes.POINTER(Config), _c_double_p, _c_int_p,
                                                ctypes.c_void_p]),
    ("xslam_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("xslam_se3_exp_compose", ctypes.c_int, [_c_double_p, _c_double_p, _c_double_p]),
    # include/xslam_plain.h: the plain FP64 complex path
    ("xslam_plain_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_float, ctypes.c_float, _c_float_p, ctypes.POINTER(Intrinsics),
                                          ctypes.POINTER(Config), ctypes.c_int, ctypes.c_void_p]),
    ("xslam_plain_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("xslam_plain_set_pose", ctypes.c_int, [ctypes.c_void_p, _c_double_p]),
    ("xslam_plain_frame", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Seed),
                                         ctypes.c_int, _c_double_p, _c_double_p, _c_double_p]),
    ("xslam_plain_read_tsdf", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("xslam_plain_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    # include/xslam_batch.h: many trajectories per step
    ("xslam_batch_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    ("xslam_batch_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("xslam_batch_step", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("xslam_batch_sync", ctypes.c_int, [ctypes.c_void_p, _c_int_p]),
    ("xslam_batch_read", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_double_p, _c_double_p, _c_double_p]),
    ("xslam_batch_latency", ctypes.c_int, [ctypes.c_void_p, _c_float_p]),
    ("xslam_batch_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _c_int_p,
                                            _c_float_p]),
    ("xslam_batch_set_shapes", ctypes.c_int, [ctypes.c_void_p, _c_int_p]),
    ("xslam_batch_profile", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("xslam_batch_profile_read", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_int_p, _c_int_p, _c_int_p,
                                                _c_float_p, _c_int_p]),
    ("xslam_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    # include/xslam_mlp.h: the learned pose proposal
    ("xslam_mlp_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _c_int_p, ctypes.c_int,
                                        ctypes.c_void_p]),
    ("xslam_mlp_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("xslam_mlp_param_count", ctypes.c_size_t, [ctypes.c_void_p]),
    ("xslam_mlp_set_params", ctypes.c_int, [ctypes.c_void_p, _c_float_p]),
    ("xslam_mlp_get_params", ctypes.c_int, [ctypes.c_void_p, _c_float_p]),
    ("xslam_mlp_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("xslam_mlp_gradient", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, _c_float_p,
                                          _c_double_p]),
    ("xslam_mlp_features", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    ("xslam_mlp_pair_targets", ctypes.c_int, [_c_double_p, ctypes.c_int, _c_int_p, ctypes.c_int, _c_float_p,
                                              _c_float_p]),
    ("xslam_mlp_train", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                       ctypes.c_ulonglong, ctypes.c_int, _c_float_p]),
    ("xslam_gemm_bf16", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("xslam_set_proposal", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _c_float_p, ctypes.c_int]),
    ("xslam_counters", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]),
    ("xslam_mlp_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
]
STAGES = ("prepare", "icp", "integrate", "raycast", "other")


def load(path: str = LIB_PATH):
    """Load libxslam.so and declare its C signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -m paper_2405_02187_gb300._build` "
                           "(or __graft_entry__.build()) on a machine with nvcc")
    lib = ctypes.CDLL(path)
    for name, res, args in SYMBOLS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def se3_exp_compose(xi, T=None):
    """exp(xi) T (3x4; T = identity when None) through the library's FP64 SE(3) exponential."""
    lib = load()
    x = np.ascontiguousarray(xi, np.float64).reshape(6)
    Tm = np.eye(3, 4) if T is None else np.asarray(T, np.float64)
    Tin = np.ascontiguousarray(Tm[:3, :4], np.float64).reshape(-1).copy()
    out = np.zeros(12)
    st = lib.xslam_se3_exp_compose(_dptr(x), _dptr(Tin), _dptr(out))
    if st != OK:
        raise XSlamError(st, "xslam_se3_exp_compose: NULL or non-finite argument")
    return out.reshape(3, 4)


def icp_system_noalloc(depth, level, intr, model, Tj, T_prev, seeds=(), cfg: Config | None = None, stream=None):
    """ICP normal equations with no allocation inside the library (see xslam_icp_system_noalloc):
    depth is the level's CUDA float32 depth, model the (1 + 6 (1 + K)) x H x W CUDA float32 maps.
    Returns ((1 + K, 27) array, n_valid)."""
    lib = load()
    K = len(seeds)
    W, H = int(intr.width), int(intr.height)
    Kin = Intrinsics(float(intr.fx), float(intr.fy), float(intr.cx), float(intr.cy), W, H)
    Tj = np.ascontiguousarray(Tj, np.float64).reshape(-1)
    T_prev = np.ascontiguousarray(T_prev, np.float64).reshape(-1)
    # the C call reads (H >> level)(W >> level) depths, (1 + 6 (1 + K)) H W model floats and
    # 12 (1 + K) doubles of each pose block: a shorter buffer would be read past its end
    if Tj.size != 12 * (1 + K) or T_prev.size != 12 * (1 + K):
        raise ValueError(f"Tj and T_prev must hold (1 + K) x 12 = {12 * (1 + K)} doubles")
    if not 0 <= int(level) <= 2:
        raise ValueError("level must be 0, 1 or 2")
    if depth is None or depth.numel() != (H >> int(level)) * (W >> int(level)):
        raise ValueError(f"depth must hold {(H >> int(level)) * (W >> int(level))} floats for level {level}")
    if model is None or model.numel() < (1 + 6 * (1 + K)) * H * W:
        raise ValueError(f"model must hold at least (1 + 6 (1 + K)) H W = {(1 + 6 * (1 + K)) * H * W} floats")
    out = np.zeros(27 * (1 + K))
    n = ctypes.c_int(0)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.xslam_icp_system_noalloc(_dev(depth), int(level), ctypes.byref(Kin), _dev(model), _dptr(Tj), _dptr(T_prev),
                                      _seeds(seeds), K, ctypes.byref(cfg) if cfg is not None else None, _dptr(out),
                                      ctypes.byref(n), ctypes.c_void_p(stream))
    if st != OK:
        raise XSlamError(st, lib.xslam_last_error(None).decode())
    return out.reshape(1 + K, 27), n.value


def default_config() -> Config:
    c = Config()
    load().xslam_default_config(ctypes.byref(c))
    return c


def _dptr(a):
    """Pointer to a float64 numpy array (contiguous)."""
    return a.ctypes.data_as(_c_double_p)


def _dev(t, dtype_name="float32"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous() or str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected a contiguous {dtype_name} CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _sym6(packed):
    """Symmetric 6x6 matrix from its packed upper triangle (row by row)."""
    H = np.zeros((6, 6))
    iu = np.triu_indices(6)
    H[iu] = packed
    H[(iu[1], iu[0])] = packed
    return H


def _seeds(seeds):
    arr = (Seed * max(1, len(seeds)))()
    for i, s in enumerate(seeds):
        kind, index, h = s
        arr[i] = Seed(int(kind), int(index), float(h))
    return arr


class XSlam:
    """One X-KinectFusion volume and its frame state (a handle of libxslam)."""

    def __init__(self, dims, voxel, trunc, origin, intr, cfg: Config | None = None, max_lanes=6, stream=None):
        self.lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.intr = intr
        self.W, self.H = int(intr.width), int(intr.height)
        K = Intrinsics(float(intr.fx), float(intr.fy), float(intr.cx), float(intr.cy), self.W, self.H)
        org = (ctypes.c_float * 3)(*[float(o) for o in origin])
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        st = self.lib.xslam_create(ctypes.byref(h), *self.dims, float(voxel), float(trunc), org, ctypes.byref(K),
                                   ctypes.byref(cfg) if cfg is not None else None, int(max_lanes),
                                   ctypes.c_void_p(stream))
        if st != OK:
            raise XSlamError(st, self.lib.xslam_last_error(None).decode())
        self.h = h
        self.K = 0
        self.max_lanes = max_lanes

    # -- helpers ---------------------------------------------------------------------------
    def _check(self, st, allow=(OK,)):
        if st not in allow:
            raise XSlamError(st, self.lib.xslam_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.xslam_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_vox(self):
        return self.dims[0] * self.dims[1] * self.dims[2]

    def _depth(self, t):
        """Device pointer of a CUDA depth map, checked to hold H x W floats (the library reads that many)."""
        if t is not None and t.numel() != self.W * self.H:
            raise ValueError(f"depth has {t.numel()} values, expected {self.H} x {self.W}")
        return _dev(t)

    def _out(self, t, n):
        """Device pointer of a CUDA output buffer, checked to hold at least n floats."""
        if t is not None and t.numel() < n:
            raise ValueError(f"output buffer has {t.numel()} values, needs {n}")
        return _dev(t)

    # -- sequence API ----------------------------------------------------------------------
    def reset(self):
        self._check(self.lib.xslam_reset(self.h))
        self.K = 0
        self._inflight = {}

    def set_pose(self, T):
        T = np.ascontiguousarray(T, np.float64).reshape(12)
        self._check(self.lib.xslam_set_pose(self.h, _dptr(T)))

    def frame(self, depth, seeds=(), outputs=True):
        """Run one frame. depth: CUDA float32 tensor (H, W) or host numpy float32 array.
        Returns (pose (3,4), dpose (K,3,4), dtwist (K,6), status) or status if outputs is False."""
        K = len(seeds)
        sd = _seeds(seeds)
        n = depth.size if isinstance(depth, np.ndarray) else depth.numel()
        if n != self.W * self.H:
            raise ValueError(f"depth has {n} values, expected {self.H} x {self.W}")
        if isinstance(depth, np.ndarray):
            depth = np.ascontiguousarray(depth, np.float32)
            ptr, on_dev = ctypes.c_void_p(depth.ctypes.data), 0
        elif not depth.is_cuda:  # a (pinned) host tensor
            assert depth.is_contiguous() and str(depth.dtype) == "torch.float32"
            ptr, on_dev = ctypes.c_void_p(depth.data_ptr()), 0
        else:
            ptr, on_dev = _dev(depth), 1
        if not outputs:
            st = self.lib.xslam_frame(self.h, ptr, on_dev, sd, K, None, None, None)
            self._check(st, (OK, ENOTRACK))
            self.K = K
            return st
        pose = np.zeros(12)
        dpose = np.zeros(max(1, 12 * K))
        dtw = np.zeros(max(1, 6 * K))
        st = self.lib.xslam_frame(self.h, ptr, on_dev, sd, K, _dptr(pose), _dptr(dpose), _dptr(dtw))
        self._check(st, (OK, ENOTRACK))
        self.K = K
        return pose.reshape(3, 4), dpose[:12 * K].reshape(K, 3, 4), dtw[:6 * K].reshape(K, 6), st

    def submit(self, depth, seeds=()):
        """Enqueue one frame without waiting (xslam_frame_submit); returns its ticket for wait(). A host
        depth map (ideally a pinned tensor) is kept referenced until its frame is waited for."""
        K = len(seeds)
        sd = _seeds(seeds)
        n = depth.size if isinstance(depth, np.ndarray) else depth.numel()
        if n != self.W * self.H:
            raise ValueError(f"depth has {n} values, expected {self.H} x {self.W}")
        if isinstance(depth, np.ndarray):
            depth = np.ascontiguousarray(depth, np.float32)
            ptr, on_dev = ctypes.c_void_p(depth.ctypes.data), 0
        elif not depth.is_cuda:
            assert depth.is_contiguous() and str(depth.dtype) == "torch.float32"
            ptr, on_dev = ctypes.c_void_p(depth.data_ptr()), 0
        else:
            ptr, on_dev = _dev(depth), 1
        t = ctypes.c_longlong(0)
        self._check(self.lib.xslam_frame_submit(self.h, ptr, on_dev, sd, K, ctypes.byref(t)))
        self.K = K
        if not hasattr(self, "_inflight"):
            self._inflight = {}
        self._inflight[t.value] = (depth, K)
        return t.value

    def wait(self, ticket):
        """Outputs of a submitted frame (xslam_frame_wait; tickets in submission order): (pose (3,4),
        dpose (K,3,4), dtwist (K,6), status)."""
        _, K = self._inflight.get(ticket, (None, self.K))
        pose = np.zeros(12)
        dpose = np.zeros(max(1, 12 * K))
        dtw = np.zeros(max(1, 6 * K))
        st = self.lib.xslam_frame_wait(self.h, int(ticket), _dptr(pose), _dptr(dpose), _dptr(dtw))
        if st in (OK, ENOTRACK, ETIMEOUT):
            self._inflight.pop(ticket, None)
        self._check(st, (OK, ENOTRACK))
        return pose.reshape(3, 4), dpose[:12 * K].reshape(K, 3, 4), dtw[:6 * K].reshape(K, 6), st

    def sync(self):
        n = ctypes.c_int(0)
        st = self._check(self.lib.xslam_sync(self.h, ctypes.byref(n)), (OK, ENOTRACK))
        return st, n.value

    def raycast(self, T=None, depth=None, vmap=None, nmap=None):
        Tp = None
        if T is not None:
            T = np.ascontiguousarray(T, np.float64).reshape(-1)
            Tp = _dptr(T)
        hw = self.W * self.H
        self._check(self.lib.xslam_raycast(self.h, Tp, self._out(depth, hw), self._out(vmap, 3 * (1 + self.K) * hw),
                                           self._out(nmap, 3 * (1 + self.K) * hw)))

    def grad(self, query_depth, T_q, order=1):
        T_q = np.ascontiguousarray(T_q, np.float64).reshape(12)
        loss = ctypes.c_double(0)
        g = np.zeros(6)
        H = np.zeros(21)
        self._check(self.lib.xslam_grad(self.h, self._depth(query_depth), _dptr(T_q), int(order), ctypes.byref(loss),
                                        _dptr(g), _dptr(H)))
        if order == 2:
            Hm = np.zeros((6, 6))
            iu = np.triu_indices(6)
            Hm[iu] = H
            Hm[(iu[1], iu[0])] = H
            return loss.value, g, Hm
        return loss.value, g

    def grad_plain64(self, query_depth, T_q):
        """(E, g[6], H[6x6]) of the order-2 loss by the plain FP64 bicomplex path (xslam_grad_plain64)."""
        T_q = np.ascontiguousarray(T_q, np.float64).reshape(12)
        loss = ctypes.c_double(0)
        g = np.zeros(6)
        H = np.zeros(21)
        self._check(self.lib.xslam_grad_plain64(self.h, self._depth(query_depth), _dptr(T_q), ctypes.byref(loss),
                                                _dptr(g), _dptr(H)))
        return loss.value, g, _sym6(H)

    def grad_tsdf(self, query_depth, T_q, order=2):
        """TSDF-difference relocalisation loss (E, g[6], H 6x6 or None, observed voxels updated) at T_q."""
        T_q = np.ascontiguousarray(T_q, np.float64).reshape(12)
        loss = ctypes.c_double(0)
        n = ctypes.c_longlong(0)
        g = np.zeros(6)
        H = np.zeros(21)
        self._check(self.lib.xslam_grad_tsdf(self.h, self._depth(query_depth), _dptr(T_q), int(order), ctypes.byref(loss),
                                             _dptr(g), _dptr(H), ctypes.byref(n)))
        Hm = None
        if order == 2:
            Hm = np.zeros((6, 6))
            iu = np.triu_indices(6)
            Hm[iu] = H
            Hm[(iu[1], iu[0])] = H
        return loss.value, g, Hm, n.value

    def grad_tsdf_plain64(self, query_depth, T_q):
        """The same (E, g, H, updated voxels) by the plain FP64 bicomplex path (full products, h = 1e-20)."""
        T_q = np.ascontiguousarray(T_q, np.float64).reshape(12)
        loss = ctypes.c_double(0)
        n = ctypes.c_longlong(0)
        g = np.zeros(6)
        H = np.zeros(21)
        self._check(self.lib.xslam_grad_tsdf_plain64(self.h, self._depth(query_depth), _dptr(T_q), ctypes.byref(loss),
                                                     _dptr(g), _dptr(H), ctypes.byref(n)))
        Hm = np.zeros((6, 6))
        iu = np.triu_indices(6)
        Hm[iu] = H
        Hm[(iu[1], iu[0])] = H
        return loss.value, g, Hm, n.value

    def read_tsdf(self, lane, out):
        self._check(self.lib.xslam_read_tsdf(self.h, int(lane), self._out(out, self.n_vox)))
        return out

    def profile(self, enable=True):
        self._check(self.lib.xslam_profile(self.h, int(bool(enable))))

    def profile_read(self):
        """dict stage -> (ms, launches), plus counters (fused voxels, ray-cast surface pixels, frames)."""
        ms = np.zeros(len(STAGES))
        la = (ctypes.c_longlong * len(STAGES))()
        c = np.zeros(3)
        self._check(self.lib.xslam_profile_read(self.h, _dptr(ms), la, _dptr(c)))
        return {s: (ms[i], la[i]) for i, s in enumerate(STAGES)}, dict(fused=c[0], hits=c[1], frames=c[2])

    # -- stage API -------------------------------------------------------------------------
    def set_lanes(self, seeds):
        sd = _seeds(seeds)
        self._check(self.lib.xslam_set_lanes(self.h, sd, len(seeds)))
        self.K = len(seeds)

    def set_pose_lanes(self, T):
        T = np.ascontiguousarray(T, np.float64).reshape(-1)
        assert T.size == 12 * (1 + self.K)
        self._check(self.lib.xslam_set_pose_lanes(self.h, _dptr(T)))

    def get_pose_lanes(self):
        T = np.zeros(12 * (1 + self.K))
        self._check(self.lib.xslam_get_pose_lanes(self.h, _dptr(T)))
        return T.reshape(1 + self.K, 3, 4)

    def write_tsdf(self, lane, t):
        self._check(self.lib.xslam_write_tsdf(self.h, int(lane), self._out(t, self.n_vox)))

    def measure(self, depth, level=0, out=None):
        n_out = (self.W >> int(level)) * (self.H >> int(level)) if 0 <= int(level) < 3 else 0
        self._check(self.lib.xslam_measure(self.h, self._depth(depth), int(level), self._out(out, n_out)))
        return out

    def integrate(self, depth):
        self._check(self.lib.xslam_integrate(self.h, self._depth(depth)))

    def set_model(self, depth, vmap, nmap, T_prev):
        T_prev = np.ascontiguousarray(T_prev, np.float64).reshape(-1)
        n_map = 3 * (1 + self.K) * self.W * self.H
        self._check(self.lib.xslam_set_model(self.h, self._depth(depth), self._out(vmap, n_map), self._out(nmap, n_map),
                                             _dptr(T_prev)))

    def set_proposal(self, mlp, scale=None, judge_level=2):
        """Attach the learned proposal (an Mlp; None detaches) with its output scale (6 values)."""
        if mlp is None:
            self._check(self.lib.xslam_set_proposal(self.h, None, None, 0))
            return
        sc = np.ascontiguousarray(scale, np.float32).reshape(6)
        self._check(self.lib.xslam_set_proposal(self.h, mlp.m, sc.ctypes.data_as(_c_float_p), int(judge_level)))
        self._proposal = mlp  # must outlive the attachment

    def counters(self, reset=False):
        """dict: ICP iterations computed, proposals judged, proposals accepted."""
        c = (ctypes.c_ulonglong * 3)()
        self._check(self.lib.xslam_counters(self.h, c, int(bool(reset))))
        return dict(icp_iterations=c[0], judged=c[1], accepted=c[2])

    def icp_system(self, level, Tj):
        Tj = np.ascontiguousarray(Tj, np.float64).reshape(-1)
        out = np.zeros(27 * (1 + self.K))
        n = ctypes.c_int(0)
        self._check(self.lib.xslam_icp_system(self.h, int(level), _dptr(Tj), _dptr(out), ctypes.byref(n)))
        return out.reshape(1 + self.K, 27), n.value


class XSlamPlain:
    """The plain FP64 complex path (include/xslam_plain.h): one complex<double> run per seed."""

    def __init__(self, dims, voxel, trunc, origin, intr, cfg: Config | None = None, max_runs=6, stream=None):
        self.lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.W, self.H = int(intr.width), int(intr.height)
        K = Intrinsics(float(intr.fx), float(intr.fy), float(intr.cx), float(intr.cy), self.W, self.H)
        org = (ctypes.c_float * 3)(*[float(o) for o in origin])
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        st = self.lib.xslam_plain_create(ctypes.byref(h), *self.dims, float(voxel), float(trunc), org, ctypes.byref(K),
                                         ctypes.byref(cfg) if cfg is not None else None, int(max_runs),
                                         ctypes.c_void_p(stream))
        if st != OK:
            raise XSlamError(st, self.lib.xslam_plain_last_error(None).decode())
        self.h = h
        self.max_runs = max_runs

    def _check(self, st, allow=(OK,)):
        if st not in allow:
            raise XSlamError(st, self.lib.xslam_plain_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.xslam_plain_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_vox(self):
        return self.dims[0] * self.dims[1] * self.dims[2]

    def _depth(self, t):
        """Device pointer of a CUDA depth map, checked to hold H x W floats (the library reads that many)."""
        if t is not None and t.numel() != self.W * self.H:
            raise ValueError(f"depth has {t.numel()} values, expected {self.H} x {self.W}")
        return _dev(t)

    def _out(self, t, n):
        """Device pointer of a CUDA output buffer, checked to hold at least n floats."""
        if t is not None and t.numel() < n:
            raise ValueError(f"output buffer has {t.numel()} values, needs {n}")
        return _dev(t)

    def set_pose(self, T):
        T = np.ascontiguousarray(T, np.float64).reshape(12)
        self._check(self.lib.xslam_plain_set_pose(self.h, _dptr(T)))

    def frame(self, depth, seeds=()):
        """Run one frame of every run; returns (pose (3,4), dpose (K,3,4), dtwist (K,6), status)."""
        K = len(seeds)
        n = depth.size if isinstance(depth, np.ndarray) else depth.numel()
        if n != self.W * self.H:
            raise ValueError(f"depth has {n} values, expected {self.H} x {self.W}")
        if isinstance(depth, np.ndarray):
            depth = np.ascontiguousarray(depth, np.float32)
            ptr, on_dev = ctypes.c_void_p(depth.ctypes.data), 0
        elif not depth.is_cuda:
            assert depth.is_contiguous() and str(depth.dtype) == "torch.float32"
            ptr, on_dev = ctypes.c_void_p(depth.data_ptr()), 0
        else:
            ptr, on_dev = _dev(depth), 1
        pose = np.zeros(12)
        dpose = np.zeros(max(1, 12 * K))
        dtw = np.zeros(max(1, 6 * K))
        st = self.lib.xslam_plain_frame(self.h, ptr, on_dev, _seeds(seeds), K, _dptr(pose), _dptr(dpose), _dptr(dtw))
        self._check(st, (OK, ENOTRACK))
        return pose.reshape(3, 4), dpose[:12 * K].reshape(K, 3, 4), dtw[:6 * K].reshape(K, 6), st

    def read_tsdf(self, run, part, out):
        """part 0: Re F, 1: Im F / h, 2: W, into a CUDA float64 tensor of nx*ny*nz."""
        self._check(self.lib.xslam_plain_read_tsdf(self.h, int(run), int(part), _dev(out, "float64")))
        return out


class XSlamBatch:
    """Several XSlam handles advanced together, one CUDA graph per step (include/xslam_batch.h).
    Every handle must be before its first frame with its lanes (set_lanes) and pose (set_pose) set."""

    def __init__(self, handles, stream=None):
        self.lib = load()
        self.handles = list(handles)  # keeps them alive
        n = len(self.handles)
        arr = (ctypes.c_void_p * n)(*[h.h for h in self.handles])
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        b = ctypes.c_void_p()
        st = self.lib.xslam_batch_create(ctypes.byref(b), n, arr, ctypes.c_void_p(stream))
        if st != OK:
            raise XSlamError(st, self.lib.xslam_batch_last_error(None).decode())
        self.b = b
        self.n = n
        self._keep = None

    def _check(self, st):
        if st != OK:
            raise XSlamError(st, self.lib.xslam_batch_last_error(self.b).decode())

    def close(self):
        if getattr(self, "b", None):
            self.lib.xslam_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptrs(self, depths):
        assert len(depths) == self.n
        return (ctypes.c_void_p * self.n)(*[None if d is None else _dev(d).value for d in depths])

    def step(self, depths):
        """depths: n CUDA float32 tensors (or None for a trajectory that does not advance)."""
        self._keep = list(depths)  # the tensors must outlive the asynchronous step
        self._check(self.lib.xslam_batch_step(self.b, self._ptrs(depths)))

    def sync(self):
        nf = (ctypes.c_int * self.n)()
        self._check(self.lib.xslam_batch_sync(self.b, nf))
        return list(nf)

    def read(self, i):
        K = self.handles[i].K
        pose = np.zeros(12)
        dpose = np.zeros(max(1, 12 * K))
        dtw = np.zeros(max(1, 6 * K))
        self._check(self.lib.xslam_batch_read(self.b, int(i), _dptr(pose), _dptr(dpose), _dptr(dtw)))
        return pose.reshape(3, 4), dpose[:12 * K].reshape(K, 3, 4), dtw[:6 * K].reshape(K, 6)

    def latency(self):
        ms = np.zeros(self.n, np.float32)
        self._check(self.lib.xslam_batch_latency(self.b, ms.ctypes.data_as(_c_float_p)))
        return ms

    def autotune(self, frames, steps):
        """frames[s][i]: CUDA depth tensor of trajectory i at step s (None = inactive)."""
        flat = []
        for s_ in range(steps):
            flat += [None if d is None else _dev(d).value for d in frames[s_]]
        arr = (ctypes.c_void_p * len(flat))(*flat)
        choice = (ctypes.c_int * 4)()
        ms = np.zeros(15, np.float32)
        self._check(self.lib.xslam_batch_autotune(self.b, arr, int(steps), choice, ms.ctypes.data_as(_c_float_p)))
        ms = ms[:int(np.count_nonzero(ms))]
        return dict(icp_divisor=choice[0], fuse_blocks_per_sm=choice[1], ray_tile=self.TILES[choice[2]],
                    mode=self.MODES[choice[3]]), ms

    TILES = ("32x8", "16x16", "64x4")
    MODES = ("segmented", "branches")

    def set_shapes(self, choice):
        """Launch shapes as autotune returns them (a dict)."""
        c = (ctypes.c_int * 4)(int(choice["icp_divisor"]), int(choice["fuse_blocks_per_sm"]),
                               self.TILES.index(choice["ray_tile"]), self.MODES.index(choice["mode"]))
        self._check(self.lib.xslam_batch_set_shapes(self.b, c))

    STAGES = ("measure", "seed", "icp", "tiles", "update", "raycast", "readout")

    def profile(self, enable=True):
        """Launch profile of the segmented step (adds an event after every launch; not for timed runs)."""
        self._check(self.lib.xslam_batch_profile(self.b, int(bool(enable))))

    def profile_read(self, cap=1024):
        """The last step's launches: list of (stage, argument, blocks, ms); empty in branch mode."""
        kind = np.zeros(cap, np.int32)
        arg = np.zeros(cap, np.int32)
        blk = np.zeros(cap, np.int32)
        ms = np.zeros(cap, np.float32)
        n = ctypes.c_int()
        self._check(self.lib.xslam_batch_profile_read(self.b, cap, kind.ctypes.data_as(_c_int_p),
                                                      arg.ctypes.data_as(_c_int_p), blk.ctypes.data_as(_c_int_p),
                                                      ms.ctypes.data_as(_c_float_p), ctypes.byref(n)))
        m = min(n.value, cap)
        return [(self.STAGES[kind[q]], int(arg[q]), int(blk[q]), float(ms[q])) for q in range(m)]


# ------------------------------------------------------------------------------------------------
# include/xslam_mlp.h: the learned pose proposal
# ------------------------------------------------------------------------------------------------
def _bf16(t):
    return _dev(t, "bfloat16")


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    return ctypes.c_void_p(stream)


def _mlp_raise(st, m=None):
    lib = load()
    raise XSlamError(st, lib.xslam_mlp_last_error(m).decode())


def features(depth, depth_min, depth_max, out=None, stream=None):
    """80 x 60 BF16 features of CUDA depth frames (n, H, W) or (H, W) into out (n, 4800)."""
    import torch
    lib = load()
    d = depth if depth.dim() == 3 else depth[None]
    n, H, W = d.shape
    if out is None:
        out = torch.empty((n, 4800), dtype=torch.bfloat16, device=d.device)
    st = lib.xslam_mlp_features(_dev(d), int(n), int(W), int(H), float(depth_min), float(depth_max), _bf16(out),
                                _stream_ptr(stream))
    if st != OK:
        _mlp_raise(st)
    return out


def pair_targets(poses, pairs, scale):
    """log(T_i^-1 T_j) / scale for each pair (host; poses (n, 3, 4), pairs (P, 2)) -> (P, 6) float32."""
    lib = load()
    poses = np.ascontiguousarray(poses, np.float64).reshape(-1, 12)
    pairs = np.ascontiguousarray(pairs, np.int32).reshape(-1, 2)
    sc = np.ascontiguousarray(scale, np.float32).reshape(6)
    out = np.zeros((pairs.shape[0], 6), np.float32)
    st = lib.xslam_mlp_pair_targets(_dptr(poses), poses.shape[0], pairs.ctypes.data_as(_c_int_p), pairs.shape[0],
                                    sc.ctypes.data_as(_c_float_p), out.ctypes.data_as(_c_float_p))
    if st != OK:
        _mlp_raise(st)
    return out


def gemm_bf16(A, B, C, splits=1, workspace=None, stream=None):
    """C = A B^T on the tensor cores (A (M, K), B (N, K) CUDA bfloat16, C (M, N) CUDA float32)."""
    lib = load()
    M, K = A.shape
    N = B.shape[0]
    st = lib.xslam_gemm_bf16(_bf16(A), _bf16(B), int(M), int(N), int(K), _dev(C), int(splits), _dev(workspace),
                             _stream_ptr(stream))
    if st != OK:
        _mlp_raise(st)
    return C


class Mlp:
    """The proposal network (xslam_mlp_t): sizes (n_0, ..., n_L), batches of up to max_batch rows."""

    def __init__(self, sizes, max_batch=256, stream=None):
        self.lib = load()
        self.sizes = tuple(int(s) for s in sizes)
        arr = (ctypes.c_int * len(self.sizes))(*self.sizes)
        m = ctypes.c_void_p()
        st = self.lib.xslam_mlp_create(ctypes.byref(m), len(self.sizes) - 1, arr, int(max_batch), _stream_ptr(stream))
        if st != OK:
            _mlp_raise(st)
        self.m = m
        self.max_batch = max_batch
        self.n_params = int(self.lib.xslam_mlp_param_count(m))

    def _check(self, st):
        if st != OK:
            _mlp_raise(st, self.m)

    def close(self):
        if getattr(self, "m", None):
            self.lib.xslam_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def flatten(params):
        """[(W (out, in), b (out)), ...] -> the flat host layout."""
        return np.concatenate([np.concatenate([np.asarray(W, np.float32).reshape(-1), np.asarray(b, np.float32)])
                               for W, b in params])

    def unflatten(self, flat):
        out, k = [], 0
        for n_in, n_out in zip(self.sizes[:-1], self.sizes[1:]):
            W = flat[k:k + n_in * n_out].reshape(n_out, n_in)
            k += n_in * n_out
            out.append((W, flat[k:k + n_out]))
            k += n_out
        return out

    def set_params(self, params):
        flat = np.ascontiguousarray(self.flatten(params) if isinstance(params, (list, tuple)) else params, np.float32)
        assert flat.size == self.n_params
        self._check(self.lib.xslam_mlp_set_params(self.m, flat.ctypes.data_as(_c_float_p)))

    def get_params(self):
        flat = np.zeros(self.n_params, np.float32)
        self._check(self.lib.xslam_mlp_get_params(self.m, flat.ctypes.data_as(_c_float_p)))
        return self.unflatten(flat)

    def forward(self, x, y=None):
        """x: CUDA bfloat16 (B, n_0) -> CUDA float32 (B, n_L)."""
        import torch
        if y is None:
            y = torch.empty((x.shape[0], self.sizes[-1]), dtype=torch.float32, device=x.device)
        self._check(self.lib.xslam_mlp_forward(self.m, _bf16(x), int(x.shape[0]), _dev(y)))
        return y

    def gradient(self, x, targets):
        """Loss and gradient (list of (dW, db)) of the batch x (CUDA bf16) with CUDA float32 targets."""
        g = np.zeros(self.n_params, np.float32)
        loss = ctypes.c_double(0)
        self._check(self.lib.xslam_mlp_gradient(self.m, _bf16(x), _dev(targets), int(x.shape[0]),
                                                g.ctypes.data_as(_c_float_p), ctypes.byref(loss)))
        return loss.value, self.unflatten(g)

    def train(self, feat, pairs, targets, epochs, batch=256, lr=1e-3, seed=1, mirror=False):
        """Adam over the pairs (CUDA int32 (P, 2)) of feature rows feat (CUDA bf16 (n, 4800)) with CUDA
        float32 targets (P, n_L), optionally with random reflections; returns the per-epoch mean loss."""
        losses = np.zeros(epochs, np.float32)
        self._check(self.lib.xslam_mlp_train(self.m, _bf16(feat), int(feat.shape[0]), _dev(pairs, "int32"),
                                             _dev(targets), int(pairs.shape[0]), int(batch), int(epochs), float(lr),
                                             int(seed), int(bool(mirror)), losses.ctypes.data_as(_c_float_p)))
        return losses
