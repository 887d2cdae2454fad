"""Thin Python binding of the C ABI in include/qmckl_gpu.h.

Argument marshalling only: every step of the evaluation runs in the CUDA
library ``libqmckl_gpu.so``.  Host arrays are numpy; device buffers and
streams come from PyTorch (``tensor.data_ptr()``, ``stream.cuda_stream``).
There is no CPU fallback: if the library is missing, loading it raises.

Usage, following the paper's example (Sec. 5.1)::

    ctx = Context(mode="bf16x3")
    ctx.set_molecule(mol)              # nuclei, shells, primitives, MOs, cutoff
    ctx.set_points_device(coord)       # [walk][elec][3] float64 CUDA tensor
    out = ctx.mo_vgl_device()          # [walk][elec][5][mo] CUDA tensor
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqmckl_gpu.so")

QK_SUCCESS = 0
STATUS_NAMES = {
    0: "QK_SUCCESS", -1: "QK_ERR_INVALID_ARG", -2: "QK_ERR_NULL_POINTER",
    -3: "QK_ERR_BAD_SIZE", -4: "QK_ERR_NOT_PROVIDED", -5: "QK_ERR_NOT_IMPLEMENTED",
    -6: "QK_ERR_CUDA", -7: "QK_ERR_DEVICE_TIMEOUT", -8: "QK_ERR_OUT_OF_MEMORY",
}
MODES = {"fp64": 0, "fp32": 1, "bf16x3": 2, "tf32": 3}

# every exported symbol with its ctypes signature (restype is qk_status unless noted)
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double
_SZ = ctypes.c_size_t
SIGNATURES = {
    "qk_context_create": [ctypes.POINTER(_P)],
    "qk_context_destroy": [_P],
    "qk_last_error": [_P, ctypes.c_char_p, _I64],
    "qk_set_precision": [_P, _I32],
    "qk_set_cutoff": [_P, _D],
    "qk_set_compute_mode": [_P, _I32],
    "qk_set_fusion": [_P, _I32],
    "qk_set_spatial_order": [_P, _I32],
    "qk_set_basis_order": [_P, _I32],
    "qk_get_basis_order": [_P, ctypes.POINTER(_I32)],
    "qk_get_shell_order": [_P, _P, _I64],
    "qk_set_mo_cusp": [_P, _P],
    "qk_get_density_device": [_P, _P, _P, _I64],
    "qk_set_single_point_device": [_P, _I64, _P],
    "qk_get_mo_vgl_single_device": [_P, _P, _I64],
    "qk_accept_single_point": [_P],
    "qk_get_mo_cusp_coefficients_device": [_P, _P, _I64],
    "qk_set_nucleus": [_P, _I64, _P, _P],
    "qk_set_ao_basis": [_P, _I64, _I64, _P, _P, _P, _P, _P, _P, _P, _I64, _P],
    "qk_set_mo_coefficient": [_P, _I64, _P],
    "qk_set_points": [_P, ctypes.c_char, _I64, _I64, _P],
    "qk_set_points_device": [_P, ctypes.c_char, _I64, _I64, _P],
    "qk_get_nucl_num": [_P, ctypes.POINTER(_I64)],
    "qk_get_ao_num": [_P, ctypes.POINTER(_I64)],
    "qk_get_mo_num": [_P, ctypes.POINTER(_I64)],
    "qk_get_point_num": [_P, ctypes.POINTER(_I64)],
    "qk_workspace_size": [_P, ctypes.POINTER(_SZ)],
    "qk_set_workspace": [_P, _P, _SZ],
    "qk_set_stream": [_P, _P],
    "qk_synchronize": [_P],
    "qk_get_ao_vgl": [_P, _P, _I64],
    "qk_get_ao_vgl_device": [_P, _P, _I64],
    "qk_get_mo_vgl": [_P, _P, _I64],
    "qk_get_mo_vgl_device": [_P, _P, _I64],
    "qk_mo_vgl_backward_device": [_P, _P, _I64, _P, _P],
    "qk_backward_workspace_size": [_P, ctypes.POINTER(_SZ)],
    "qk_set_timing": [_P, _I32],
    "qk_get_kernel_count": [_P, ctypes.POINTER(_I64)],
    "qk_get_block_stats": [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                           ctypes.POINTER(_I64)],
    "qk_get_sparsity_stats": [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "qk_get_tile_layout": [_P, _P, _I64, _P, _I64, _P, _I64],
    "qk_get_ao_chunk_num": [_P, ctypes.POINTER(_I64)],
    "qk_set_sm_pairs": [_P, _I32],
    "qk_batch_create": [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P)],
    "qk_batch_destroy": [_P],
    "qk_batch_last_error": [_P, ctypes.c_char_p, _I64],
    "qk_batch_set_stream": [_P, _P],
    "qk_batch_set_graph": [_P, _I32],
    "qk_batch_set_sm_pairs": [_P, _I32],
    "qk_batch_set_tile": [_P, _I32],
    "qk_batch_get_tile": [_P, ctypes.POINTER(_I32)],
    "qk_batch_run": [_P, ctypes.POINTER(_P), ctypes.POINTER(_I64)],
    "qk_batch_synchronize": [_P],
    "qk_batch_autotune": [_P, ctypes.POINTER(_P), _I32, ctypes.POINTER(_D)],
    "qk_contract_device": [_I32, _I64, _I64, _I64, _P, _P, _P, _P],
    "qk_contract_device_noalloc": [_I32, _I64, _I64, _I64, _P, _P, _P, _P],
    "qk_selftest_wait_timeout": [_I64, _P],
    "qk_get_timing": [_P, ctypes.POINTER(_D), ctypes.POINTER(_I64), _I32],
}

_lib = None


class QmcklError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with paper_2512_16677_gb300.build() "
                "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int32
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _tptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _device_tensor(t, what, dtype=None, numel=None, min_numel=None):
    """Check a tensor handed to the library by pointer: on the GPU,
    contiguous, of the element type the library reads or writes, and (where
    the C call takes no size) of the element count it touches."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what}: a CUDA tensor is required")
    if not t.is_contiguous():
        raise ValueError(f"{what}: the tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{what}: dtype {t.dtype}, expected {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what}: {t.numel()} elements, expected {numel}")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{what}: {t.numel()} elements, at least {min_numel} needed")
    return t


def contract_device(A, B, mode: str = "fp32", out=None):
    """D = A @ B.T on the GPU with the kernel of `mode` (CUDA tensors)."""
    import torch
    lib = load()
    M, K = A.shape
    N = B.shape[0]
    dt = torch.float64 if mode == "fp64" else torch.float32
    _device_tensor(A, "A", dt)
    _device_tensor(B, "B", dt, numel=N * K)
    if out is None:
        out = torch.empty((M, N), dtype=dt, device=A.device)
    _device_tensor(out, "out", dt, numel=M * N)
    st = lib.qk_contract_device(MODES[mode], M, N, K, _tptr(A), _tptr(B), _tptr(out),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != QK_SUCCESS:
        raise QmcklError(st, "qk_contract_device")
    return out


class Context:
    """One QMCkl-style context (not thread-safe; use one per thread)."""

    def __init__(self, mode: str = "fp64"):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.qk_context_create(ctypes.byref(h))
        if st != QK_SUCCESS:
            raise QmcklError(st, "qk_context_create failed")
        self.h = h
        self._ws = None
        self._keep = []
        self._walk_elec_shape = (0, 0)
        self.charges = None
        self.mode = mode
        self.set_compute_mode(mode)

    # ----------------------------------------------------------- plumbing
    def _check(self, st: int, what: str):
        if st != QK_SUCCESS:
            buf = ctypes.create_string_buffer(512)
            self.lib.qk_last_error(self.h, buf, 512)
            raise QmcklError(st, f"{what}: {buf.value.decode(errors='replace')}")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.qk_context_destroy(self.h)
            self.h = ctypes.c_void_p()
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ settings
    def set_precision(self, bits: int):
        self._check(self.lib.qk_set_precision(self.h, bits), "set_precision")

    def set_cutoff(self, eps: float):
        self._check(self.lib.qk_set_cutoff(self.h, eps), "set_cutoff")

    def set_fusion(self, enable: bool):
        """split-bf16: build AO blocks inside the contraction kernel (default
        off: ao_vgl and the contraction run as two kernels)."""
        self._check(self.lib.qk_set_fusion(self.h, 1 if enable else 0), "set_fusion")

    def set_mo_cusp(self, rc):
        """Cusp radii [nucl] in bohr (None switches the correction off)."""
        if rc is None:
            self._check(self.lib.qk_set_mo_cusp(self.h, None), "set_mo_cusp")
            return
        a = _f64(rc)
        self._check(self.lib.qk_set_mo_cusp(self.h, _ptr(a)), "set_mo_cusp")

    def cusp_coefficients_device(self):
        """f [nucl][mo][4] (FP64 CUDA tensor) of the current cusp correction."""
        import torch
        self._bind_stream()
        n = self.lib
        nn, nm = self.nucl_num, self.mo_num
        out = torch.empty((nn, nm, 4), dtype=torch.float64, device="cuda")
        self._check(n.qk_get_mo_cusp_coefficients_device(self.h, out.data_ptr(), out.numel()),
                    "get_mo_cusp_coefficients_device")
        return out

    def set_single_point_device(self, elec: int, coords):
        """Proposed positions [walk][3] (CUDA float64) of electron `elec`."""
        import torch
        _device_tensor(coords, "coords", torch.float64, numel=3 * self._walk_elec()[0])
        self._bind_stream()
        self._single = coords  # kept alive until the copy has run
        self._check(self.lib.qk_set_single_point_device(self.h, int(elec), coords.data_ptr()),
                    "set_single_point_device")

    def mo_vgl_single_device(self, out=None):
        """MO vgl [walk][5][mo] at the proposed positions (CUDA tensor)."""
        import torch
        w = self._walk_elec()[0]
        if out is None:
            out = torch.empty((w, 5, self.mo_num), dtype=self.dtype_torch, device="cuda")
        _device_tensor(out, "out", self.dtype_torch)
        self._bind_stream()
        self._check(self.lib.qk_get_mo_vgl_single_device(self.h, out.data_ptr(), out.numel()),
                    "get_mo_vgl_single_device")
        return out

    def accept_single_point(self):
        self._bind_stream()
        self._check(self.lib.qk_accept_single_point(self.h), "accept_single_point")

    def density_device(self, w, out=None):
        """Electron density sum_i w_i phi_i^2 at the current points as a CUDA
        tensor [point_num] (FP64 in fp64 mode, else FP32)."""
        import torch
        wa = _f64(w)
        if wa.shape != (self.mo_num,):
            raise ValueError("one occupation weight per MO")
        n = self.point_num
        dt = torch.float64 if self.mode == "fp64" else torch.float32
        if out is None:
            out = torch.empty(n, dtype=dt, device="cuda")
        _device_tensor(out, "out", dt)
        self._bind_stream()
        self._check(self.lib.qk_get_density_device(self.h, _ptr(wa), out.data_ptr(), out.numel()),
                    "get_density_device")
        return out

    def set_basis_order(self, mode: int):
        """0: nuclei order chosen from the geometry (default), 1: caller's
        shell order, 2: nuclei in Morton order; 0 and 2 then split the shells
        into compact and diffuse classes.  Applies to the next set_molecule /
        basis."""
        self._check(self.lib.qk_set_basis_order(self.h, int(mode)), "set_basis_order")

    def basis_order_spatial(self) -> bool:
        """Whether the current basis takes its nuclei in Morton order."""
        v = ctypes.c_int32()
        self._check(self.lib.qk_get_basis_order(self.h, ctypes.byref(v)), "get_basis_order")
        return bool(v.value)

    def shell_order(self, shell_num: int) -> np.ndarray:
        """The caller's shell at each internal position."""
        out = np.zeros(shell_num, dtype=np.int64)
        self._check(self.lib.qk_get_shell_order(self.h, _ptr(out), shell_num),
                    "get_shell_order")
        return out

    def set_sm_pairs(self, enable: bool):
        """Contraction on pairs of SMs (default) or on single SMs."""
        self._check(self.lib.qk_set_sm_pairs(self.h, 1 if enable else 0), "set_sm_pairs")

    def set_spatial_order(self, enable: bool):
        """tensor-core modes: cut point tiles from a spatial order (default on)."""
        self._check(self.lib.qk_set_spatial_order(self.h, 1 if enable else 0),
                    "set_spatial_order")

    def set_compute_mode(self, mode: str):
        self._check(self.lib.qk_set_compute_mode(self.h, MODES[mode]), "set_compute_mode")
        self.mode = mode

    @property
    def dtype_np(self):
        return np.float64 if self.mode == "fp64" else np.float32

    @property
    def dtype_torch(self):
        import torch
        return torch.float64 if self.mode == "fp64" else torch.float32

    # -------------------------------------------------------------- system
    def set_nucleus(self, charge, coord):
        charge, coord = _f64(charge), _f64(coord).reshape(-1, 3)
        self.charges = charge
        self._check(self.lib.qk_set_nucleus(self.h, charge.shape[0], _ptr(charge), _ptr(coord)),
                    "set_nucleus")

    def set_ao_basis(self, shell_nucleus, shell_ang_mom, shell_prim_num, shell_factor,
                     exponent, coefficient, prim_factor, ao_factor):
        sn = np.ascontiguousarray(shell_nucleus, dtype=np.int64)
        sl = np.ascontiguousarray(shell_ang_mom, dtype=np.int32)
        sp = np.ascontiguousarray(shell_prim_num, dtype=np.int64)
        sf, ex, co, pf, af = map(_f64, (shell_factor, exponent, coefficient, prim_factor,
                                        ao_factor))
        self._check(self.lib.qk_set_ao_basis(
            self.h, sn.shape[0], ex.shape[0], _ptr(sn), _ptr(sl), _ptr(sp), _ptr(sf), _ptr(ex),
            _ptr(co), _ptr(pf), af.shape[0], _ptr(af)), "set_ao_basis")

    def set_mo_coefficient(self, C):
        C = _f64(C)
        self._check(self.lib.qk_set_mo_coefficient(self.h, C.shape[0], _ptr(C)),
                    "set_mo_coefficient")

    def set_molecule(self, mol, points: bool = False):
        """Nuclei, basis, MO coefficients and cutoff of a synth.Molecule."""
        self.set_nucleus(mol.nucl_charge, mol.nucl_coord)
        self.set_ao_basis(mol.shell_nucleus, mol.shell_ang_mom, mol.shell_prim_num,
                          mol.shell_factor, mol.exponent, mol.coefficient, mol.prim_factor,
                          mol.ao_factor)
        self.set_mo_coefficient(mol.mo_coef)
        if getattr(mol, "eps", None) is not None:
            self.set_cutoff(mol.eps)
        else:
            self.set_precision(int(mol.bits))
        if points:
            self.set_points(mol.coord)

    # -------------------------------------------------------------- points
    def set_points(self, coord, transp: str = "N"):
        """Host coordinates [walk][elec][3] ('N') or [3][walk*elec] ('T')."""
        c = _f64(coord)
        if transp == "N":
            w, e = (c.shape[0], c.shape[1]) if c.ndim == 3 else (1, c.size // 3)
        else:
            w, e = 1, c.size // 3
        self._check(self.lib.qk_set_points(self.h, transp.encode(), w, e, _ptr(c)), "set_points")
        self._walk_elec_shape = (w, e)

    def set_points_device(self, coord, transp: str = "N", walk_num=None, elec_num=None):
        """CUDA float64 tensor [walk][elec][3] (or [3][n] with transp='T')."""
        if walk_num is None:
            if transp == "N":
                walk_num, elec_num = (coord.shape[0], coord.shape[1]) if coord.dim() == 3 \
                    else (1, coord.shape[0])
            else:
                walk_num, elec_num = 1, coord.numel() // 3
        import torch
        _device_tensor(coord, "coord", torch.float64, min_numel=3 * walk_num * elec_num)
        self._bind_stream()
        self._keep = [coord]
        self._check(self.lib.qk_set_points_device(self.h, transp.encode(), walk_num, elec_num,
                                                  _tptr(coord)), "set_points_device")
        self._walk_elec_shape = (walk_num, elec_num)

    # --------------------------------------------------------------- sizes
    def _get_i64(self, fn, what):
        v = ctypes.c_int64()
        self._check(fn(self.h, ctypes.byref(v)), what)
        return v.value

    @property
    def nucl_num(self):
        return self._get_i64(self.lib.qk_get_nucl_num, "get_nucl_num")

    @property
    def ao_num(self):
        return self._get_i64(self.lib.qk_get_ao_num, "get_ao_num")

    @property
    def mo_num(self):
        return self._get_i64(self.lib.qk_get_mo_num, "get_mo_num")

    @property
    def point_num(self):
        return self._get_i64(self.lib.qk_get_point_num, "get_point_num")

    # ----------------------------------------------------- device plumbing
    def _bind_stream(self):
        import torch
        self._check(self.lib.qk_set_stream(self.h, ctypes.c_void_p(
            torch.cuda.current_stream().cuda_stream)), "set_stream")

    def workspace_size(self) -> int:
        v = ctypes.c_size_t()
        self._check(self.lib.qk_workspace_size(self.h, ctypes.byref(v)), "workspace_size")
        return v.value

    def backward_workspace_size(self) -> int:
        v = ctypes.c_size_t()
        self._check(self.lib.qk_backward_workspace_size(self.h, ctypes.byref(v)),
                    "backward_workspace_size")
        return v.value

    def ensure_workspace(self, extra: int = 0):
        """Caller-owned workspace from the torch allocator (grown as needed)."""
        import torch
        need = self.workspace_size() + extra
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            off = (-base) % 256
            self._check(self.lib.qk_set_workspace(self.h, ctypes.c_void_p(base + off),
                                                  need + 256 - off), "set_workspace")
        return self._ws

    def set_timing(self, enable: bool):
        self._check(self.lib.qk_set_timing(self.h, 1 if enable else 0), "set_timing")

    def get_timing(self):
        """(ms per class, launches per class) for ao_vgl, contraction, other."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int64 * 3)()
        self._check(self.lib.qk_get_timing(self.h, ms, n, 3), "get_timing")
        return list(ms), list(n)

    def synchronize(self):
        self._check(self.lib.qk_synchronize(self.h), "synchronize")

    def block_stats(self):
        """(live blocks, all blocks, live (point, AO) entries) of the current
        AO tensor in a tensor-core mode."""
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.qk_get_block_stats(self.h, ctypes.byref(a), ctypes.byref(b),
                                                ctypes.byref(c)), "get_block_stats")
        return a.value, b.value, c.value

    def kernel_count(self) -> int:
        """Kernel launches of the timed classes since the last call (then reset)."""
        v = ctypes.c_int64()
        self._check(self.lib.qk_get_kernel_count(self.h, ctypes.byref(v)), "get_kernel_count")
        return v.value

    def sparsity_stats(self):
        """(live (tile, 16-AO group) pairs, nonzero (point, AO) pairs) of the
        current AO tensor on the two-kernel tensor-core path."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.qk_get_sparsity_stats(self.h, ctypes.byref(a), ctypes.byref(b)),
                    "get_sparsity_stats")
        return a.value, b.value

    def tile_layout(self, groups: bool = False):
        """(perm, live[, groups]): the caller's point at each slot of the
        contraction tiles (25 slots per tile), the live AO blocks of each
        tile and, with groups=True, the [tile][chunk] bit masks of live
        16-AO column groups, for the AO tensor of the current points
        (tensor-core path)."""
        n = self.point_num
        tiles = (n + 24) // 25
        perm = np.zeros(n, dtype=np.int32)
        live = np.zeros(tiles, dtype=np.int32)
        nchunk = 0
        g = None
        if groups:
            nchunk = self._get_i64(self.lib.qk_get_ao_chunk_num, "get_ao_chunk_num")
            g = np.zeros((tiles, nchunk), dtype=np.uint8)
        self._check(self.lib.qk_get_tile_layout(
            self.h, perm.ctypes.data, n, live.ctypes.data, tiles,
            None if g is None else g.ctypes.data, 0 if g is None else g.size),
            "get_tile_layout")
        return (perm, live, g) if groups else (perm, live)

    # ------------------------------------------------------------ evaluate
    def mo_vgl_device(self, out=None):
        """MO vgl [walk][elec][5][mo] as a CUDA tensor (async on torch's stream)."""
        import torch
        w, e = self._walk_elec()
        if out is None:
            out = torch.empty((w, e, 5, self.mo_num), dtype=self.dtype_torch, device="cuda")
        _device_tensor(out, "out", self.dtype_torch)
        self._bind_stream()
        self.ensure_workspace()
        self._check(self.lib.qk_get_mo_vgl_device(self.h, _tptr(out), out.numel()),
                    "get_mo_vgl_device")
        return out

    def backward_device(self, dW, need_dC: bool = True, need_dR: bool = True):
        """(dL/dC [mo][ao], dL/dR [nucl][3]) as CUDA float64 tensors for
        L = sum(dW * mo_vgl) at the current points (async on torch's stream)."""
        import torch
        _device_tensor(dW, "dW", self.dtype_torch)
        self._bind_stream()
        self.ensure_workspace(extra=self.backward_workspace_size())
        dC = torch.empty((self.mo_num, self.ao_num), dtype=torch.float64, device="cuda") \
            if need_dC else None
        dR = torch.empty((self.nucl_num, 3), dtype=torch.float64, device="cuda") \
            if need_dR else None
        self._check(self.lib.qk_mo_vgl_backward_device(
            self.h, _tptr(dW), dW.numel(), _tptr(dC) if dC is not None else None,
            _tptr(dR) if dR is not None else None), "mo_vgl_backward_device")
        return dC, dR

    def ao_vgl_device(self, out=None):
        import torch
        w, e = self._walk_elec()
        if out is None:
            out = torch.empty((w, e, 5, self.ao_num), dtype=self.dtype_torch, device="cuda")
        _device_tensor(out, "out", self.dtype_torch)
        self._bind_stream()
        self._check(self.lib.qk_get_ao_vgl_device(self.h, _tptr(out), out.numel()),
                    "get_ao_vgl_device")
        return out

    def mo_vgl(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        """MO vgl into host memory (blocking)."""
        n = self.point_num * 5 * self.mo_num
        if out is None:
            out = np.empty(n, dtype=self.dtype_np)
        self._check(self.lib.qk_get_mo_vgl(self.h, _ptr(out), out.size), "get_mo_vgl")
        return out.reshape(self.point_num, 5, self.mo_num)

    def ao_vgl(self) -> np.ndarray:
        n = self.point_num * 5 * self.ao_num
        out = np.empty(n, dtype=self.dtype_np)
        self._check(self.lib.qk_get_ao_vgl(self.h, _ptr(out), out.size), "get_ao_vgl")
        return out.reshape(self.point_num, 5, self.ao_num)

    def _walk_elec(self):
        return self._walk_elec_shape


class Batch:
    """Several contexts (molecules of uneven sizes) evaluated by two
    persistent launches captured in a CUDA graph (qk_batch_* calls)."""

    def __init__(self, contexts):
        self.lib = load()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        h = ctypes.c_void_p()
        for c in self.contexts:
            c.ensure_workspace()
        st = self.lib.qk_batch_create(ctypes.byref(h), len(self.contexts), arr)
        if st != QK_SUCCESS:
            raise QmcklError(st, "qk_batch_create: contexts must be set and share a "
                                 "tensor-core mode")
        self.h = h
        self._outs = None

    def _check(self, st, what):
        if st != QK_SUCCESS:
            buf = ctypes.create_string_buffer(512)
            self.lib.qk_batch_last_error(self.h, buf, 512)
            raise QmcklError(st, f"{what}: {buf.value.decode(errors='replace')}")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.qk_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind_stream(self):
        import torch
        self._check(self.lib.qk_batch_set_stream(self.h, ctypes.c_void_p(
            torch.cuda.current_stream().cuda_stream)), "set_stream")

    def set_graph(self, enable: bool):
        self._check(self.lib.qk_batch_set_graph(self.h, 1 if enable else 0), "set_graph")

    def set_sm_pairs(self, enable: bool):
        self._check(self.lib.qk_batch_set_sm_pairs(self.h, 1 if enable else 0), "set_sm_pairs")

    def set_tile(self, bn_max: int):
        self._check(self.lib.qk_batch_set_tile(self.h, bn_max), "set_tile")

    @property
    def tile(self) -> int:
        v = ctypes.c_int32()
        self._check(self.lib.qk_batch_get_tile(self.h, ctypes.byref(v)), "get_tile")
        return v.value

    def outputs(self):
        """One float32 CUDA tensor [walk][elec][5][mo] per context (kept)."""
        import torch
        if self._outs is None:
            self._outs = [torch.empty((c._walk_elec_shape[0], c._walk_elec_shape[1], 5, c.mo_num),
                                      dtype=torch.float32, device="cuda")
                          for c in self.contexts]
        return self._outs

    def _ptrs(self, outs):
        return (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])

    def run(self, outs=None):
        import torch
        outs = self.outputs() if outs is None else outs
        for o in outs:
            _device_tensor(o, "batch output", torch.float32)
        self._bind_stream()
        sizes = (ctypes.c_int64 * len(outs))(*[o.numel() for o in outs])
        self._check(self.lib.qk_batch_run(self.h, self._ptrs(outs), sizes), "batch_run")
        return outs

    def synchronize(self):
        self._check(self.lib.qk_batch_synchronize(self.h), "batch_synchronize")

    def autotune(self, reps: int = 3):
        """Time every instantiated tile width on this batch; keep the fastest.
        Returns (bn_max, ms per contraction launch)."""
        self._bind_stream()
        best = ctypes.c_double()
        self._check(self.lib.qk_batch_autotune(self.h, self._ptrs(self.outputs()), reps,
                                               ctypes.byref(best)), "batch_autotune")
        return self.tile, best.value
