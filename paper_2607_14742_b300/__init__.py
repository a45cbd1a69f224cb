"""Python binding of libcare_b300.so, the B300 (sm_103a) mixed-precision CARE solver.

Thin marshalling over the C ABI declared in include/care_b300.h: tensors are
passed by device pointer, PyTorch supplies device memory (the solver
workspace included) and the current CUDA stream.  Every computation runs in
the library's CUDA kernels and host control code; there is no Python or CPU
fallback -- if the shared library is missing or no CUDA device is present the
calls raise.

Boundary layout: matrices are float64 column-major in the C ABI.  Here B
(n x m), C (p x n), W (n x b) and the returned Z (n x r) are ordinary torch
tensors in their mathematical shapes; the binding transposes to/from the
column-major storage the library expects.  The kernel-level calls (spmm, gram)
take row-major blocks, the library's internal layout.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcare_b300.so")

PREC_FP64 = 0
PREC_MIXED_FP32 = 1
PREC_MIXED_TF32 = 2
PREC_MIXED_BF16 = 3
PREC = {"fp64": PREC_FP64, "mixed": PREC_MIXED_FP32, "mixed_fp32": PREC_MIXED_FP32, "mixed_tf32": PREC_MIXED_TF32,
        "mixed_bf16": PREC_MIXED_BF16}
KRYLOV_BICGSTAB = 0
KRYLOV_GMRES = 1
KRYLOV_DENSE_LU = 2
DENSE_LU_MAX_N = 8192
PRECOND_NONE = 0
PRECOND_JACOBI = 1
PRECOND_ILU0 = 2
PRECOND_ILU0_EXACT = 3
HIST_MAX = 32


class CareError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class csr_t(ct.Structure):
    _fields_ = [("n", ct.c_int), ("nnz", ct.c_int), ("rowptr", ct.c_void_p), ("colind", ct.c_void_p),
                ("val", ct.c_void_p)]


class opts_t(ct.Structure):
    _fields_ = [("kmax", ct.c_int), ("jmax", ct.c_int), ("newton_max", ct.c_int), ("adi_cap", ct.c_int),
                ("eta_r_rel", ct.c_double), ("eta_s_mult", ct.c_double), ("tau_L_lo", ct.c_double),
                ("tau_L_hi", ct.c_double), ("tau_N_lo", ct.c_double), ("tau_N_hi", ct.c_double),
                ("krylov_tol_lo", ct.c_double), ("krylov_tol_hi", ct.c_double),
                ("krylov_maxit_lo", ct.c_int), ("krylov_maxit_hi", ct.c_int), ("krylov", ct.c_int),
                ("precond", ct.c_int), ("krylov_chunk", ct.c_int), ("stag_ratio", ct.c_double),
                ("shift_hmin", ct.c_int), ("ilu_sweeps", ct.c_int), ("tri_sweeps", ct.c_int),
                ("verbose", ct.c_int), ("inner_compress", ct.c_int), ("gmres_restart_lo", ct.c_int),
                ("gmres_restart_hi", ct.c_int)]


class info_t(ct.Structure):
    _fields_ = [("status", ct.c_int), ("rank", ct.c_int), ("iter0_outer", ct.c_int), ("iter0_inner", ct.c_int),
                ("iter_outer", ct.c_int), ("iter_inner", ct.c_int), ("krylov_iters", ct.c_longlong),
                ("spmm_calls", ct.c_longlong), ("krylov_unconverged", ct.c_int), ("nhist", ct.c_int),
                ("res_hist", ct.c_double * HIST_MAX), ("res_rel_CtC", ct.c_double), ("res_paper", ct.c_double),
                ("ms_phase", ct.c_double * 4), ("ms_total", ct.c_double),
                ("gram_ms", ct.c_double * 2), ("gram_gflop", ct.c_double * 2), ("gram_calls", ct.c_longlong * 2),
                ("gemm_ms", ct.c_double * 2), ("gemm_gflop", ct.c_double * 2), ("gemm_calls", ct.c_longlong * 2),
                ("tc_ms", ct.c_double * 2), ("tc_gflop", ct.c_double * 2), ("tc_calls", ct.c_longlong * 2),
                ("krylov_ms", ct.c_double), ("krylov_gbyte", ct.c_double), ("host_syncs", ct.c_longlong),
                ("lowp_gram_calls", ct.c_longlong)]


class op_t(ct.Structure):
    _fields_ = [("n", ct.c_int), ("nnz", ct.c_int), ("rowptr_t", ct.c_void_p), ("colind_t", ct.c_void_p),
                ("val64_t", ct.c_void_p), ("val32_t", ct.c_void_p), ("diag64", ct.c_void_p),
                ("diag32", ct.c_void_p), ("rowsum32_t", ct.c_void_p), ("max_row_nnz", ct.c_int),
                ("diag_const", ct.c_int), ("full_diag", ct.c_int),
                ("a_fro", ct.c_double)]


_lib = None


def lib() -> ct.CDLL:
    """Load libcare_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not built: run `python -m paper_2607_14742_b300.build`")
    L = ct.CDLL(LIB_PATH)
    vp, i, d, sz = ct.c_void_p, ct.c_int, ct.c_double, ct.c_size_t
    P = ct.POINTER
    sig = {
        "care_opts_default": (None, [P(opts_t)]),
        "care_status_string": (ct.c_char_p, [i]),
        "care_version": (ct.c_char_p, []),
        "care_op_size": (i, [i, i, P(sz)]),
        "care_op_prepare": (i, [P(csr_t), vp, sz, vp, P(op_t)]),
        "care_spmm": (i, [P(op_t), i, i, d, d, vp, i, i, vp, i, vp]),
        "care_gram_work_size": (sz, [i, i, i]),
        "care_gram": (i, [i, i, i, i, vp, i, vp, i, vp, i, vp, sz, vp]),
        "care_gram_noalloc": (i, [i, i, i, i, vp, i, vp, i, vp, i, vp]),
        "care_shifted_solve_workspace_size": (i, [P(op_t), i, i, i, P(opts_t), P(sz)]),
        "care_shifted_solve": (i, [P(op_t), vp, i, vp, i, i, d, d, vp, i, i, i, P(opts_t), vp, i, vp, sz, vp,
                                   P(i)]),
        "care_workspace_size": (i, [i, i, i, i, i, i, P(opts_t), P(sz)]),
        "care_solve": (i, [P(csr_t), vp, i, i, vp, i, i, d, i, P(opts_t), vp, i, i, vp, sz, vp, P(info_t)]),
        "lyap_lradi": (i, [P(csr_t), vp, i, vp, i, i, vp, i, i, d, i, P(opts_t), vp, i, i, vp, sz, vp, P(info_t)]),
        "care_residual_factor": (i, [P(csr_t), vp, i, i, vp, i, i, vp, i, i, d, vp, i, P(i), vp, i, P(i), i, P(d),
                                     vp, sz, vp]),
        "care_workspace_size_batched": (i, [i, vp, vp, vp, vp, i, P(opts_t), i, P(sz)]),
        "care_solve_batched": (i, [i, vp, vp, vp, vp, vp, vp, vp, d, i, P(opts_t), vp, vp, vp, i, vp, sz, vp, vp]),
        "care_workspace_size_batched_persistent": (i, [i, vp, vp, vp, vp, i, P(opts_t), P(sz)]),
        "care_solve_batched_persistent": (i, [i, vp, vp, vp, vp, vp, vp, vp, d, i, P(opts_t), vp, vp, vp, vp, sz,
                                              vp, vp, P(ct.c_longlong)]),
        "care_autotune_workspace_size": (i, [P(op_t), i, i, i, P(sz)]),
        "care_autotune": (i, [P(op_t), i, i, i, P(opts_t), vp, sz, vp, P(d)]),
        "care_kernel_launches": (ct.c_ulonglong, []),
        "care_fp64_peak": (i, [P(d), vp]),
        "care_symeig_work_size": (sz, [i]),
        "care_get_launch_shape": (i, [vp, P(i), P(i)]),
        "care_set_launch_shape": (i, [i, i, i]),
        "care_ilu0_work_size": (sz, [P(op_t), i]),
        "care_ilu0": (i, [P(op_t), i, i, d, d, vp, vp, sz, vp]),
        "care_symeig": (i, [i, vp, i, vp, vp, d, d, P(i), vp, sz, vp]),
        "care_tc_available": (i, []),
        "care_set_tensor_cores": (None, [i]),
        "care_tc_test_starve": (None, [i]),
        "care_tc_work_size": (sz, [i]),
        "care_gram_tc": (i, [i, i, i, i, vp, i, vp, i, vp, i, vp, sz, vp]),
        "care_gemm_ts": (i, [i, i, i, i, i, d, vp, i, vp, i, d, vp, i, vp, sz, vp]),
        "care_host_symeig": (i, [i, vp, vp, vp]),
        "care_host_symeig_outside": (i, [i, vp, vp, vp, d, d]),
        "care_host_cholesky_upper": (i, [i, vp, vp]),
        "care_host_pivoted_cholesky": (i, [i, vp, d, i, vp, vp, P(i)]),
        "care_host_upper_inverse": (i, [i, vp, vp]),
        "care_host_sym_lmax": (i, [i, vp, P(d)]),
        "care_host_gemm_nt": (i, [i, i, i, vp, i, vp, i, vp, vp, i, i]),
        "care_host_eigvals": (i, [i, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().care_kernel_launches())


def status_string(s: int) -> str:
    return lib().care_status_string(int(s)).decode()


def version() -> str:
    return lib().care_version().decode()


def _check(st, where, ok=(0,)):
    if st not in ok:
        raise CareError(st, where)
    return st


def default_options(**kw) -> opts_t:
    o = opts_t()
    lib().care_opts_default(ct.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t):
    return ct.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ct.c_void_p(0)


def _stream():
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_f64(x, device):
    return torch.as_tensor(x, dtype=torch.float64, device=device)


def _colmajor(M, device):
    """Column-major float64 storage of a 2D matrix: returns (tensor, ld)."""
    M = _dev_f64(M, device)
    return M.t().contiguous(), M.shape[0]


@dataclass
class CSR:
    """A (not A^T) in CSR on the device: int32 rowptr/colind, float64 values."""
    n: int
    rowptr: torch.Tensor
    colind: torch.Tensor
    val: torch.Tensor

    @property
    def nnz(self):
        return int(self.val.numel())

    @staticmethod
    def from_arrays(n, rowptr, colind, val, device="cuda"):
        return CSR(int(n), torch.as_tensor(rowptr, dtype=torch.int32, device=device).contiguous(),
                   torch.as_tensor(colind, dtype=torch.int32, device=device).contiguous(),
                   torch.as_tensor(val, dtype=torch.float64, device=device).contiguous())

    def c(self):
        return csr_t(self.n, self.nnz, self.rowptr.data_ptr(), self.colind.data_ptr(), self.val.data_ptr())


def _info_dict(inf: info_t) -> dict:
    return dict(status=status_string(inf.status), status_code=inf.status, rank=inf.rank,
                iter0=(inf.iter0_outer, inf.iter0_inner), iter=(inf.iter_outer, inf.iter_inner),
                krylov_iters=inf.krylov_iters, spmm_calls=inf.spmm_calls,
                krylov_unconverged=inf.krylov_unconverged, res_hist=list(inf.res_hist[:inf.nhist]),
                res_rel_CtC=inf.res_rel_CtC, res_paper=inf.res_paper, ms_phase=list(inf.ms_phase),
                ms_total=inf.ms_total, gram_ms=list(inf.gram_ms), gram_gflop=list(inf.gram_gflop),
                gram_calls=list(inf.gram_calls), gemm_ms=list(inf.gemm_ms), gemm_gflop=list(inf.gemm_gflop),
                gemm_calls=list(inf.gemm_calls), tc_ms=list(inf.tc_ms), tc_gflop=list(inf.tc_gflop), tc_calls=list(inf.tc_calls),
                krylov_ms=inf.krylov_ms, krylov_gbyte=inf.krylov_gbyte, host_syncs=inf.host_syncs,
                lowp_gram_calls=inf.lowp_gram_calls)


class Workspace:
    """Reusable device workspace (a uint8 torch tensor) grown on demand."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes: int, device) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != torch.device(device):
            self.buf = None
            torch.cuda.empty_cache()
            self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        return self.buf


_ws = Workspace()


def workspace_size(n, nnz, m, p, r_cap, prec="mixed", opts=None) -> int:
    o = opts or default_options()
    out = ct.c_size_t(0)
    _check(lib().care_workspace_size(n, nnz, m, p, r_cap, PREC[prec] if isinstance(prec, str) else prec,
                                     ct.byref(o), ct.byref(out)), "care_workspace_size")
    return out.value


def care_solve(A: CSR, B, C, tol=1e-10, prec="mixed", r_cap=512, opts=None, workspace: Workspace | None = None,
               allow=(0,)):
    """Solve A^T X + X A - X B B^T X + C^T C = 0, X ~ Z Z^T (Framework 1).

    Returns (Z, info): Z is an (n x rank) float64 tensor (a view of the
    column-major output buffer), info a dict of the care_info fields."""
    L = lib()
    dev = A.val.device
    o = opts or default_options()
    pc = PREC[prec] if isinstance(prec, str) else prec
    Bc, ldb = _colmajor(B, dev)
    Cc, ldc = _colmajor(C, dev)
    n, m = Bc.shape[1], Bc.shape[0]
    p = Cc.shape[1]
    assert n == A.n and Cc.shape[0] == A.n
    nbytes = workspace_size(n, A.nnz, m, p, r_cap, pc, o)
    ws = (workspace or _ws).get(nbytes, dev)
    Zc = torch.empty(r_cap, n, dtype=torch.float64, device=dev)
    inf = info_t()
    a = A.c()
    st = L.care_solve(ct.byref(a), _ptr(Bc), ldb, m, _ptr(Cc), ldc, p, float(tol), pc, ct.byref(o), _ptr(Zc), n,
                      r_cap, _ptr(ws), ws.numel(), _stream(), ct.byref(inf))
    _check(st, "care_solve", ok=tuple(allow) + (0,))
    return Zc[:inf.rank].t(), _info_dict(inf)


def care_solve_batched(problems, tol=1e-10, prec="mixed", r_cap=256, opts=None, workers=4, allow=(0,),
                       persistent=False, stats=None):
    """Solve independent CAREs together.  problems: list of (A: CSR, B, C).
    persistent=False: care_solve_batched (host workers, bitwise equal to single
    solves); True: care_solve_batched_persistent (shifted solves of all instances
    in shared persistent launches; stats["batch_launches"] receives their count).
    Returns (list of Z, list of info dicts, status)."""
    L = lib()
    o = opts or default_options()
    pc = PREC[prec] if isinstance(prec, str) else prec
    cnt = len(problems)
    keep = []
    csrs = (csr_t * cnt)()
    Ap = (ct.POINTER(csr_t) * cnt)()
    Bp, Cp, Zp = (ct.c_void_p * cnt)(), (ct.c_void_p * cnt)(), (ct.c_void_p * cnt)()
    ldb, ldc, ldz = (ct.c_int * cnt)(), (ct.c_int * cnt)(), (ct.c_int * cnt)()
    ms, ps, rc = (ct.c_int * cnt)(), (ct.c_int * cnt)(), (ct.c_int * cnt)()
    Zs = []
    dev = problems[0][0].val.device if cnt else "cuda"
    for i, (A, B, C) in enumerate(problems):
        Bc, lb = _colmajor(B, A.val.device)
        Cc, lc = _colmajor(C, A.val.device)
        keep += [Bc, Cc]
        csrs[i] = A.c()
        Ap[i] = ct.pointer(csrs[i])
        Bp[i], Cp[i] = Bc.data_ptr(), Cc.data_ptr()
        ldb[i], ldc[i] = lb, Cc.shape[1]
        ms[i], ps[i] = Bc.shape[0], Cc.shape[1]
        rc[i] = r_cap
        Zc = torch.empty(r_cap, A.n, dtype=torch.float64, device=A.val.device)
        Zs.append(Zc)
        Zp[i], ldz[i] = Zc.data_ptr(), A.n
    need = ct.c_size_t(0)
    if persistent:
        _check(L.care_workspace_size_batched_persistent(cnt, Ap, ms, ps, rc, pc, ct.byref(o), ct.byref(need)),
               "care_workspace_size_batched_persistent")
    else:
        _check(L.care_workspace_size_batched(cnt, Ap, ms, ps, rc, pc, ct.byref(o), workers, ct.byref(need)),
               "care_workspace_size_batched")
    ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=dev)
    infos = (info_t * cnt)()
    if persistent:
        nl = ct.c_longlong(0)
        st = L.care_solve_batched_persistent(cnt, Ap, Bp, ldb, ms, Cp, ldc, ps, float(tol), pc, ct.byref(o), Zp, ldz,
                                             rc, _ptr(ws), ws.numel(), _stream(), infos, ct.byref(nl))
        if stats is not None:
            stats["batch_launches"] = nl.value
            stats["workspace_bytes"] = need.value
    else:
        st = L.care_solve_batched(cnt, Ap, Bp, ldb, ms, Cp, ldc, ps, float(tol), pc, ct.byref(o), Zp, ldz, rc,
                                  workers, _ptr(ws), ws.numel(), _stream(), infos)
    _check(st, "care_solve_batched", ok=tuple(allow) + (0,))
    out_info = [_info_dict(infos[i]) for i in range(cnt)]
    return [Zs[i][:infos[i].rank].t() for i in range(cnt)], out_info, st


def lyap_lradi(A: CSR, W, B=None, K=None, tol=1e-10, prec="fp64", r_cap=1024, opts=None, allow=(0,)):
    """LR-ADI for (A - B K^T)^T X + X (A - B K^T) + W W^T = 0, X ~ Z Z^T."""
    L = lib()
    dev = A.val.device
    o = opts or default_options()
    o.adi_cap = max(o.adi_cap, r_cap)
    pc = PREC[prec] if isinstance(prec, str) else prec
    Wc, ldw = _colmajor(W, dev)
    b = Wc.shape[0]
    n = A.n
    if B is not None and K is not None:
        Bc, ldb = _colmajor(B, dev)
        Kc, ldk = _colmajor(K, dev)
        m = Bc.shape[0]
    else:
        Bc = Kc = None
        ldb = ldk = n
        m = 0
    nbytes = workspace_size(n, A.nnz, max(m, 1), b, r_cap, pc, o)
    ws = _ws.get(nbytes, dev)
    Zc = torch.empty(r_cap, n, dtype=torch.float64, device=dev)
    inf = info_t()
    a = A.c()
    st = L.lyap_lradi(ct.byref(a), _ptr(Bc), ldb, _ptr(Kc), ldk, m, _ptr(Wc), ldw, b, float(tol), pc, ct.byref(o),
                      _ptr(Zc), n, r_cap, _ptr(ws), ws.numel(), _stream(), ct.byref(inf))
    _check(st, "lyap_lradi", ok=tuple(allow) + (0,))
    return Zc[:inf.rank].t(), _info_dict(inf)


def care_residual_factor(A: CSR, B, C, Z, eta_r_rel=1e-4, c_cap=None):
    """Algorithm 1 in FP64: returns (C_plus, C_minus, ||R(Z Z^T)||_F)."""
    L = lib()
    dev = A.val.device
    Bc, ldb = _colmajor(B, dev)
    Cc, ldc = _colmajor(C, dev)
    Zc, ldz = _colmajor(Z, dev)
    n, m, p, r = A.n, Bc.shape[0], Cc.shape[1], Zc.shape[0]
    c_cap = c_cap or (2 * r + m + p)
    nbytes = workspace_size(n, A.nnz, m, p, max(r, 1), PREC_FP64)
    ws = _ws.get(nbytes, dev)
    Cp = torch.empty(c_cap, n, dtype=torch.float64, device=dev)
    Cm = torch.empty(c_cap, n, dtype=torch.float64, device=dev)
    rp, rm, res = ct.c_int(0), ct.c_int(0), ct.c_double(0)
    a = A.c()
    _check(L.care_residual_factor(ct.byref(a), _ptr(Bc), ldb, m, _ptr(Cc), ldc, p, _ptr(Zc), n, r,
                                  float(eta_r_rel), _ptr(Cp), n, ct.byref(rp), _ptr(Cm), n, ct.byref(rm), c_cap,
                                  ct.byref(res), _ptr(ws), ws.numel(), _stream()), "care_residual_factor")
    return Cp[:rp.value].t(), Cm[:rm.value].t(), res.value


class Operator:
    """Prepared operator (A^T in CSR, FP64 + FP32 values) living in a torch buffer."""

    def __init__(self, A: CSR):
        L = lib()
        sz = ct.c_size_t(0)
        _check(L.care_op_size(A.n, A.nnz, ct.byref(sz)), "care_op_size")
        self.mem = torch.empty(sz.value, dtype=torch.uint8, device=A.val.device)
        self.op = op_t()
        self.A = A
        a = A.c()
        _check(L.care_op_prepare(ct.byref(a), _ptr(self.mem), sz.value, _stream(), ct.byref(self.op)),
               "care_op_prepare")

    @property
    def n(self):
        return self.op.n


def spmm(op: Operator, X: torch.Tensor, shift=0.0, out: torch.Tensor | None = None):
    """Y = (A^T + shift I) X for a row-major (n x b) float32/float64/complex block X."""
    cplx = X.is_complex()
    if cplx:
        Xr = torch.view_as_real(X)  # n x b x 2
        dtype = Xr.dtype
        Xf = Xr.reshape(X.shape[0], -1)
    else:
        dtype = X.dtype
        Xf = X
    assert Xf.is_contiguous()
    vec = 2 if dtype == torch.float64 else 4
    w = Xf.shape[1]
    ld = ((w + vec - 1) // vec) * vec
    if ld != w:
        Xp = torch.zeros(Xf.shape[0], ld, dtype=dtype, device=Xf.device)
        Xp[:, :w] = Xf
    else:
        Xp = Xf
    Yp = torch.empty_like(Xp)
    b = X.shape[1]
    s = complex(shift)
    _check(lib().care_spmm(ct.byref(op.op), 0 if dtype == torch.float64 else 1, int(cplx), s.real, s.imag,
                           _ptr(Xp), ld, b, _ptr(Yp), ld, _stream()), "care_spmm")
    Y = Yp[:, :w]
    if cplx:
        Y = torch.view_as_complex(Y.reshape(X.shape[0], b, 2).contiguous())
    return Y


def autotune(op: Operator, m: int, b: int, prec="mixed", opts=None):
    """care_autotune: returns (tuned options, best shifted-solve time in ms)."""
    L = lib()
    o = opts or default_options()
    pc = PREC[prec] if isinstance(prec, str) else prec
    sz = ct.c_size_t(0)
    _check(L.care_autotune_workspace_size(ct.byref(op.op), m, b, pc, ct.byref(sz)), "care_autotune_workspace_size")
    ws = torch.empty(sz.value, dtype=torch.uint8, device=op.A.val.device)
    best = ct.c_double(0)
    _check(L.care_autotune(ct.byref(op.op), m, b, pc, ct.byref(o), _ptr(ws), ws.numel(), _stream(), ct.byref(best)),
           "care_autotune")
    return o, best.value


def gram(X: torch.Tensor, Y: torch.Tensor):
    """G = X^T Y (float64 a x b) for row-major float32/float64 blocks."""
    assert X.dtype == Y.dtype and X.shape[0] == Y.shape[0]
    n, a = X.shape
    b = Y.shape[1]
    G = torch.empty(a, b, dtype=torch.float64, device=X.device)
    ws = torch.empty(max(lib().care_gram_work_size(n, a, b), 8), dtype=torch.uint8, device=X.device)
    _check(lib().care_gram(0 if X.dtype == torch.float64 else 1, n, a, b, _ptr(X), X.stride(0), _ptr(Y),
                           Y.stride(0), _ptr(G), b, _ptr(ws), ws.numel(), _stream()), "care_gram")
    return G


TC_MODES = {"f64": 0, "tf32": 1, "bf16": 2, "f32": 3}


def launch_shape():
    """(SpMM vectors per thread per width class (5-tuple), CTAs per SM, SpMM contiguous row
    blocks) of the row-block kernels."""
    v = (ct.c_int * 5)()
    c, b = ct.c_int(0), ct.c_int(0)
    lib().care_get_launch_shape(v, ct.byref(c), ct.byref(b))
    return tuple(v), c.value, b.value


def set_launch_shape(spmm_vpt: int, ctas_per_sm: int, spmm_blocked: int = 0):
    _check(lib().care_set_launch_shape(int(spmm_vpt), int(ctas_per_sm), int(spmm_blocked)),
           "care_set_launch_shape")


def ilu0(op: Operator, shift, exact=True, dtype=torch.float64):
    """ILU(0) factor of (A + shift I)^T on A^T's pattern: a tensor of nnz values
    (complex for complex shifts) in the order of the prepared operator's rows."""
    s = complex(shift)
    cplx = s.imag != 0
    nnz = op.op.nnz
    F = torch.empty(nnz * (2 if cplx else 1), dtype=dtype, device=op.mem.device)
    dt = 0 if dtype == torch.float64 else 1
    ws = torch.empty(lib().care_ilu0_work_size(ct.byref(op.op), dt), dtype=torch.uint8, device=op.mem.device)
    _check(lib().care_ilu0(ct.byref(op.op), dt, int(bool(exact)), s.real, s.imag, _ptr(F), _ptr(ws), ws.numel(),
                           _stream()), "care_ilu0")
    return torch.view_as_complex(F.view(-1, 2)) if cplx else F


def symeig(A: torch.Tensor, lo=None, hi=None):
    """Device symmetric eigendecomposition of a float64 (n x n) tensor: returns (w
    ascending as numpy, V selected eigenvectors as rows, n_sel); eigenvectors for
    w <= lo or w >= hi (default: all)."""
    import numpy as np
    n = A.shape[0]
    A = A.contiguous()
    w = np.zeros(n)
    V = torch.empty(n, n, dtype=torch.float64, device=A.device)
    ws = torch.empty(lib().care_symeig_work_size(n), dtype=torch.uint8, device=A.device)
    ns = ct.c_int(0)
    lo = float("inf") if lo is None else float(lo)
    hi = float("-inf") if hi is None else float(hi)
    _check(lib().care_symeig(n, _ptr(A), n, w.ctypes.data, _ptr(V), lo, hi, ct.byref(ns), _ptr(ws), ws.numel(),
                             _stream()), "care_symeig")
    return w, V[:ns.value], ns.value


def fp64_peak() -> float:
    """Measured FP64 FMA throughput of the CUDA cores (TFLOP/s)."""
    t = ct.c_double(0)
    _check(lib().care_fp64_peak(ct.byref(t), _stream()), "care_fp64_peak")
    return t.value


def tc_available() -> bool:
    """True on an sm_103 device (tcgen05 + TMA)."""
    return bool(lib().care_tc_available())


def set_tensor_cores(mode):
    """Solver use of the FP64-accurate tensor-core products: 0 off, 1 where
    profitable (default), 2 every FP64 product (tests)."""
    lib().care_set_tensor_cores(int(mode))


def gram_tc(X: torch.Tensor, Y: torch.Tensor, mode="f64"):
    """G = X^T Y (float64 a x b) on the tensor cores: mode "f64" (float64 inputs,
    FP64-accurate BF16 slices), "f32" (float32 inputs, FP32-accurate slices), "tf32"
    or "bf16" (float32 inputs)."""
    assert X.dtype == Y.dtype and X.shape[0] == Y.shape[0]
    md = TC_MODES[mode]
    assert X.dtype == (torch.float64 if md == 0 else torch.float32)
    n, a = X.shape
    b = Y.shape[1]
    G = torch.empty(a, b, dtype=torch.float64, device=X.device)
    ws = torch.empty(lib().care_tc_work_size(a + b), dtype=torch.uint8, device=X.device)
    _check(lib().care_gram_tc(md, n, a, b, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0), _ptr(G), b, _ptr(ws),
                              ws.numel(), _stream()), "care_gram_tc")
    return G


def gemm_ts(X: torch.Tensor, S: torch.Tensor, alpha=1.0, beta=0.0, Y: torch.Tensor | None = None, tc=False):
    """Y = alpha X S + beta Y for row-major X (n x a), S (a x b, float64); tc=True runs
    the sliced tensor-core path (FP64-accurate for float64 X, Y; FP32-accurate for
    float32)."""
    n, a = X.shape
    b = S.shape[1]
    S = S.to(torch.float64).contiguous()
    if Y is None:
        Y = torch.zeros(n, b, dtype=X.dtype, device=X.device)
    ws = torch.empty(lib().care_tc_work_size(a + b) if tc else 8, dtype=torch.uint8, device=X.device)
    _check(lib().care_gemm_ts(0 if X.dtype == torch.float64 else 1, int(bool(tc)), n, a, b, float(alpha), _ptr(X),
                              X.stride(0), _ptr(S), S.stride(0), float(beta), _ptr(Y), Y.stride(0), _ptr(ws),
                              ws.numel(), _stream()), "care_gemm_ts")
    return Y


GRAM_NOALLOC_SCRATCH_DOUBLES = 1048576


def gram_noalloc(X: torch.Tensor, Y: torch.Tensor, out: torch.Tensor | None = None):
    """G = X^T Y through the allocation-free entry point (no workspace; the library's
    fixed device scratch).  `out` (float64 a x b) may be preallocated by the caller."""
    assert X.dtype == Y.dtype and X.shape[0] == Y.shape[0]
    n, a = X.shape
    b = Y.shape[1]
    G = out if out is not None else torch.empty(a, b, dtype=torch.float64, device=X.device)
    _check(lib().care_gram_noalloc(0 if X.dtype == torch.float64 else 1, n, a, b, _ptr(X), X.stride(0), _ptr(Y),
                                   Y.stride(0), _ptr(G), G.stride(0), _stream()), "care_gram_noalloc")
    return G


def shifted_solve(op: Operator, W, shift, B=None, K=None, prec="fp64", opts=None, with_status=False):
    """V = ((A - B K^T)^T + shift I)^{-1} W (SMW + the shifted-solve method of opts).
    Returns (V, iters), or (V, iters, status) with with_status (0 ok, 7 inner failure)."""
    L = lib()
    dev = op.A.val.device
    o = opts or default_options()
    pc = PREC[prec] if isinstance(prec, str) else prec
    Wc, ldw = _colmajor(W, dev)
    b = Wc.shape[0]
    n = op.n
    if B is not None and K is not None:
        Bc, ldb = _colmajor(B, dev)
        Kc, ldk = _colmajor(K, dev)
        m = Bc.shape[0]
    else:
        Bc = Kc = None
        ldb = ldk = n
        m = 0
    sz = ct.c_size_t(0)
    _check(L.care_shifted_solve_workspace_size(ct.byref(op.op), max(m, 1), b, pc, ct.byref(o), ct.byref(sz)),
           "care_shifted_solve_workspace_size")
    ws = torch.empty(sz.value, dtype=torch.uint8, device=dev)
    s = complex(shift)
    cplx = s.imag != 0
    Vc = torch.empty(b, n, dtype=torch.complex128 if cplx else torch.float64, device=dev)
    it = ct.c_int(0)
    st = L.care_shifted_solve(ct.byref(op.op), _ptr(Bc), ldb, _ptr(Kc), ldk, m, s.real, s.imag, _ptr(Wc), ldw, b,
                              pc, ct.byref(o), _ptr(Vc), n, _ptr(ws), ws.numel(), _stream(), ct.byref(it))
    _check(st, "care_shifted_solve", ok=(0, 7))
    return (Vc.t(), it.value, st) if with_status else (Vc.t(), it.value)


def host_symeig(A):
    """Host symmetric eigendecomposition (library routine): returns (w ascending, V)."""
    import numpy as np
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    _check(lib().care_host_symeig(n, A.ctypes.data, w.ctypes.data, V.ctypes.data), "care_host_symeig")
    return w, V


def host_symeig_outside(A, lo, hi):
    """Host symmetric eigendecomposition with eigenvectors only for w <= lo or w >= hi
    (library routine): returns (w ascending, V with zero columns elsewhere)."""
    import numpy as np
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    w = np.zeros(n)
    V = np.ones((n, n), order="F")
    _check(lib().care_host_symeig_outside(n, A.ctypes.data, w.ctypes.data, V.ctypes.data, float(lo), float(hi)),
           "care_host_symeig_outside")
    return w, V


def host_cholesky_upper(G):
    """Upper Cholesky factor R (G = R^T R) of an SPD matrix (library routine)."""
    import numpy as np
    G = np.asfortranarray(np.asarray(G, dtype=np.float64))
    n = G.shape[0]
    R = np.zeros((n, n), order="F")
    _check(lib().care_host_cholesky_upper(n, G.ctypes.data, R.ctypes.data), "care_host_cholesky_upper")
    return R


def host_pivoted_cholesky(G, tol, max_rank=0):
    """Rank-revealing pivoted Cholesky (library routine): returns (piv, R) with
    G ~= R^T R, R rank x c in the original column order."""
    import numpy as np
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64))
    c = G.shape[0]
    piv = np.zeros(max(c, 1), dtype=np.int32)
    R = np.zeros((c, c))
    rank = ct.c_int(0)
    _check(lib().care_host_pivoted_cholesky(c, G.ctypes.data, float(tol), int(max_rank), piv.ctypes.data,
                                            R.ctypes.data, ct.byref(rank)), "care_host_pivoted_cholesky")
    return piv[:rank.value], R[:rank.value]


def host_sym_lmax(G):
    """Largest eigenvalue of a symmetric matrix (library routine, Lanczos)."""
    import numpy as np
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64))
    out = ct.c_double(0.0)
    _check(lib().care_host_sym_lmax(G.shape[0], G.ctypes.data, ct.byref(out)), "care_host_sym_lmax")
    return out.value


def host_upper_inverse(U):
    """Inverse of an upper triangular matrix (library routine)."""
    import numpy as np
    U = np.ascontiguousarray(np.asarray(U, dtype=np.float64))
    r = U.shape[0]
    Ui = np.zeros((r, r))
    _check(lib().care_host_upper_inverse(r, U.ctypes.data, Ui.ctypes.data), "care_host_upper_inverse")
    return Ui


def host_gemm_nt(A, B, d=None, sym=False):
    """C = A diag(d) B^T for row-major blocks (library routine); sym: B is A."""
    import numpy as np
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    B = A if sym else np.ascontiguousarray(np.asarray(B, dtype=np.float64))
    m, k = A.shape
    n = B.shape[0]
    C = np.full((m, n), np.nan)
    dd = None if d is None else np.ascontiguousarray(np.asarray(d, dtype=np.float64))
    _check(lib().care_host_gemm_nt(m, n, k, A.ctypes.data, max(k, 1), B.ctypes.data, max(k, 1),
                                   None if dd is None else dd.ctypes.data, C.ctypes.data, max(n, 1), int(sym)),
           "care_host_gemm_nt")
    return C


def host_eigvals(A):
    """Host eigenvalues of a general real matrix (library routine)."""
    import numpy as np
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    wr = np.zeros(n)
    wi = np.zeros(n)
    _check(lib().care_host_eigvals(n, A.ctypes.data, wr.ctypes.data, wi.ctypes.data), "care_host_eigvals")
    return wr + 1j * wi
