"""Python binding of the learned prior (``sepso_prior_*``) and of the tensor-core
GEMM (``sepso_gemm_bf16``) -- argument marshalling only; every step runs in the
CUDA library.

The prior is a small MLP that maps a scene (occupancy raster + start/target) to a
proposed path, used beside Priori Initialization (Sec. 3.3.3) to seed a cycle's
particles; the paper itself has no learned component.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import check_prior


def _dev(device=None) -> torch.device:
    if not torch.cuda.is_available():
        raise RuntimeError("the SEPSO prior needs a CUDA device (there is no CPU path)")
    return torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())


def _f32(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, np.float32))
    return a.reshape(shape) if shape is not None else a


class Prior:
    """MLP x (g*g raster + start/target) -> hidden1 -> hidden2 -> 2T with BF16
    tensor-core kernels, FP32 masters and Adam; dataset rows held on the device."""

    def __init__(self, T: int = 20, grid: int = 64, hidden1: int = 1024, hidden2: int = 512,
                 max_batch: int = 1024, capacity: int = 4096, max_circles: int = 1024,
                 map_w: float = 400.0, map_h: float = 400.0, lr: float = 1e-3, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8, device=None):
        self.device = _dev(device)
        self.cfg = _native.PriorConfig(T=T, grid=grid, hidden1=hidden1, hidden2=hidden2,
                                       max_batch=max_batch, capacity=capacity, max_circles=max_circles,
                                       map_w=map_w, map_h=map_h, lr=lr, beta1=beta1, beta2=beta2, eps=eps)
        self.T, self.grid, self.H1, self.H2 = T, grid, hidden1, hidden2
        self.K = (grid * grid + 4 + 7) // 8 * 8
        self.O = 2 * T
        self.capacity, self.max_batch = capacity, max_batch
        L = _native.lib()
        size = ctypes.c_size_t()
        check_prior(L.sepso_prior_workspace_size(ctypes.byref(self.cfg), ctypes.byref(size)))
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        check_prior(L.sepso_prior_create(ctypes.byref(self.cfg), ctypes.c_void_p(self.workspace.data_ptr()),
                                         size.value, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _native.lib().sepso_prior_destroy(h)
            self._h = None

    @property
    def num_params(self) -> int:
        return int(_native.lib().sepso_prior_num_params(self._h))

    def set_params(self, params) -> None:
        p = _f32(params, (self.num_params,))
        check_prior(_native.lib().sepso_prior_set_params(self._h, _native.fptr(p)))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.num_params, np.float32)
        check_prior(_native.lib().sepso_prior_get_params(self._h, _native.fptr(p)))
        return p

    def add_scenes(self, first: int, points, circles, waypoints=None) -> None:
        """Rasterise scenes into rows [first, first + n); circles: list of (O, 3)."""
        pts = _f32(points).reshape(-1, 4)
        n = pts.shape[0]
        counts = np.array([np.asarray(c).reshape(-1, 3).shape[0] for c in circles], np.int32)
        assert counts.size == n
        flat = _f32(np.concatenate([np.asarray(c, np.float32).reshape(-1, 3) for c in circles])
                    if n else np.zeros((0, 3), np.float32))
        wp = None if waypoints is None else _f32(waypoints, (n, self.O))
        check_prior(_native.lib().sepso_prior_add_scenes(
            self._h, first, n, _native.fptr(pts), counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            _native.fptr(flat) if flat.size else None, _native.fptr(wp)))

    def get_rows(self, first: int, n: int):
        f = np.empty((n, self.K), np.float32)
        y = np.empty((n, self.O), np.float32)
        check_prior(_native.lib().sepso_prior_get_rows(self._h, first, n, _native.fptr(f), _native.fptr(y)))
        return f, y

    def forward(self, first: int, n: int) -> np.ndarray:
        y = np.empty((n, self.O), np.float32)
        check_prior(_native.lib().sepso_prior_forward(self._h, first, n, _native.fptr(y)))
        return y

    def grad(self, first: int, n: int):
        g = np.empty(self.num_params, np.float32)
        loss = np.zeros(1, np.float32)
        check_prior(_native.lib().sepso_prior_grad(self._h, first, n, _native.fptr(g), _native.fptr(loss)))
        return g, float(loss[0])

    def train(self, steps: int, batch: int, n_rows: int | None = None, first: int = -1, seed: int = 0,
              losses: bool = True):
        """Adam steps on minibatches drawn from rows [0, n_rows) (or the fixed rows
        [first, first + batch)); returns the per-step losses when asked."""
        out = np.empty(steps, np.float32) if losses else None
        nr = self.capacity if n_rows is None else n_rows
        check_prior(_native.lib().sepso_prior_train(self._h, nr, first, steps, batch, seed,
                                                    _native.fptr(out)))
        return out

    def infer(self, first: int, n: int, out: torch.Tensor | None = None) -> torch.Tensor:
        """Proposed waypoints of rows [first, first + n) into a device tensor (n, >= 2T)."""
        if out is None:
            out = torch.empty((n, self.O), dtype=torch.float32, device=self.device)
        assert out.is_cuda and out.dtype == torch.float32 and out.dim() == 2 and out.shape[0] >= n
        assert out.stride(1) == 1
        check_prior(_native.lib().sepso_prior_infer(self._h, first, n, ctypes.c_void_p(out.data_ptr()),
                                                    out.stride(0)))
        return out

    def sync(self) -> None:
        check_prior(_native.lib().sepso_prior_sync(self._h))

    def launch_count(self) -> int:
        return int(_native.lib().sepso_prior_launch_count(self._h))


def gemm_bf16(A: torch.Tensor, B: torch.Tensor, alpha: float = 1.0, bias: torch.Tensor | None = None,
              relu: bool = False, mask: torch.Tensor | None = None, out_f32: bool = True,
              out_bf16: bool = False, sync: bool = True):
    """C = epilogue(alpha * A @ B^T) on the tensor cores; A (M, K), B (N, K) BF16 CUDA."""
    assert A.is_cuda and B.is_cuda and A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16
    assert A.stride(1) == 1 and B.stride(1) == 1 and A.shape[1] == B.shape[1]
    M, K = A.shape
    N = B.shape[0]
    Cf = torch.empty((M, N), dtype=torch.float32, device=A.device) if out_f32 else None
    Cb = torch.empty((M, N), dtype=torch.bfloat16, device=A.device) if out_bf16 else None
    vp = ctypes.c_void_p
    stream = torch.cuda.current_stream(A.device).cuda_stream
    check_prior(_native.lib().sepso_gemm_bf16(
        vp(A.data_ptr()), vp(B.data_ptr()), M, N, K, A.stride(0), B.stride(0), float(alpha),
        vp(bias.data_ptr()) if bias is not None else None, int(relu),
        vp(mask.data_ptr()) if mask is not None else None, mask.stride(0) if mask is not None else 0,
        vp(Cf.data_ptr()) if Cf is not None else None, N, vp(Cb.data_ptr()) if Cb is not None else None, N,
        vp(stream)))
    if sync:
        check_prior(_native.lib().sepso_gemm_bf16_sync(vp(stream)))
    return Cf, Cb
