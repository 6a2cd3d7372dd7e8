"""ctypes binding of the C ABI in ``include/ndgf.h`` (argument marshalling only).

Every function keeps the C name and raises ``NDError`` on a non-OK status.
Array arguments may be torch tensors (CUDA or CPU) or numpy arrays (host);
complex arrays are complex128 (interleaved re, im).  The C functions see raw
pointers only, so the binding checks what they cannot: element types and
sizes of the buffers against the plan and the handle, contiguous outputs, and
real (not complex) Hamiltonian values (``_need``, ``require_real``).  ``stream=None`` means
torch's current CUDA stream.  The library is loaded from the in-tree build
``_lib/libndgf.so``; there is no fallback when it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

STATUS = {0: "ND_OK", 1: "ND_ERR_INVALID_ARG", 2: "ND_ERR_NOT_SYMMETRIC", 3: "ND_ERR_SINGULAR",
          4: "ND_ERR_NOT_SKEW_HERMITIAN", 5: "ND_ERR_OOM", 6: "ND_ERR_CUDA", 7: "ND_ERR_TIMEOUT",
          8: "ND_ERR_UNSUPPORTED"}
ND_PREC_FP64 = 0
ND_PREC_MIXED = 1
ND_PREC_FP32X2 = 2
ND_FACT_PHONON = 1
ND_FACT_TILE_LARGE = 2
ND_FACT_TILE_SMALL = 4
ND_FACT_GEMM_TC = 8
ND_FACT_GEMM_ALU = 16
ND_FACT_ADJOINT = 32
ND_FACT_GRAPH = 64
ND_FACT_TILE_XL = 128

EXPORTS = ["nd_analyze", "nd_plan_query", "nd_plan_tree", "nd_plan_cluster_sites", "nd_plan_destroy",
           "nd_fact_create", "nd_fact_destroy", "nd_factor", "nd_diag_green", "nd_certificate", "nd_fact_status",
           "nd_density", "nd_profile", "nd_invert_c64_noalloc",
           "nd_lead_create", "nd_lead_sigma", "nd_lead_status", "nd_lead_destroy", "nd_contact_current", "nd_density_gradient", "nd_profile_launches", "nd_sigma_lesser_fermi", "nd_phonon_const", "nd_phonon_scba",
           "nd_check_factor_inputs", "nd_check_lesser_inputs", "nd_selected_entries", "nd_fact_density", "nd_fact_set_wait_limit", "nd_fact_get_choice", "nd_fact_set_choice", "nd_autotune", "nd_density_jvp", "nd_poisson_create",
           "nd_poisson_apply", "nd_poisson_solve", "nd_poisson_destroy", "nd_vec_dot", "nd_vec_axpby", "nd_vec_mul", "nd_vec_scale_pos",
           "nd_last_error",
           "nd_version"]


class NDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class nd_graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p),
                ("n_contacts", ctypes.c_int32), ("contact_ptr", ctypes.c_void_p), ("contact_idx", ctypes.c_void_p),
                ("coord_dim", ctypes.c_int32), ("coords", ctypes.c_void_p)]


class nd_opts(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("split_permille", ctypes.c_int32), ("slab", ctypes.c_int32),
                ("delay", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class nd_kernel_stats(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int32), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class nd_tune_info(ctypes.Structure):
    _fields_ = [("ms_default", ctypes.c_double), ("ms_tuned", ctypes.c_double), ("gemm_steps", ctypes.c_int32),
                ("changed", ctypes.c_int32), ("passes", ctypes.c_int32), ("by_kind", ctypes.c_int32 * 5)]


class nd_plan_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("n_clusters", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("max_n", ctypes.c_int32), ("max_b", ctypes.c_int32),
                ("n_contacts", ctypes.c_int32), ("n_roots", ctypes.c_int32), ("flops_factor", ctypes.c_double),
                ("flops_green_r", ctypes.c_double), ("flops_green_lesser", ctypes.c_double),
                ("arena_bytes_fp64", ctypes.c_double), ("arena_bytes_fp32", ctypes.c_double)]


_LIB = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double


def lib():
    """Load the library (raises when it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build it with paper_1305_1070_gb300.build.build()")
        L = ctypes.CDLL(_build.LIB)
        sig = {
            "nd_analyze": ([ctypes.POINTER(nd_graph), ctypes.POINTER(nd_opts), ctypes.POINTER(_P)], _I32),
            "nd_plan_query": ([_P, ctypes.POINTER(nd_plan_info)], _I32),
            "nd_plan_tree": ([_P, _P, _P, _P, _P, _P], _I32),
            "nd_plan_cluster_sites": ([_P, _I32, _P], _I32),
            "nd_plan_destroy": ([_P], None),
            "nd_fact_create": ([_P, _I32, _I32, _I32, ctypes.POINTER(_P)], _I32),
            "nd_fact_destroy": ([_P], None),
            "nd_factor": ([_P, _P, _P, _P, _P, _I32, _D, _P], _I32),
            "nd_diag_green": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], _I32),
            "nd_fact_status": ([_P, ctypes.POINTER(_I32)], _I32),
            "nd_fact_set_wait_limit": ([_P, _I64], _I32),
            "nd_fact_get_choice": ([_P, _P, _I32, _P], _I32),
            "nd_fact_set_choice": ([_P, _P, _I32], _I32),
            "nd_autotune": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _I32, _D, _I32, _P, _P], _I32),
            "nd_certificate": ([_P, _P, _P], _I32),
            "nd_selected_entries": ([_P, _P, _P, _I32, _P, _P, _P, _P, _P], _I32),
            "nd_density": ([_P, _P, _I32, _I32, _D, _I32, _P, _P], _I32),
            "nd_fact_density": ([_P, _P, _D, _I32, _P, _P], _I32),
            "nd_invert_c64_noalloc": ([_P, _I32, _I32, _P, _P], _I32),
            "nd_profile": ([_P, _I32, _P, _I32, ctypes.POINTER(_I32)], _I32),
            "nd_lead_create": ([_I32, _I32, _P, _P, _P, ctypes.POINTER(_P)], _I32),
            "nd_lead_sigma": ([_P, _P, _I32, _D, _P, _I64, _I64, _P], _I32),
            "nd_lead_status": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)], _I32),
            "nd_contact_current": ([_P, _I32, _P, _P, _P], _I32),
            "nd_density_gradient": ([_P, _P, _P, _P], _I32),
            "nd_density_jvp": ([_P, _P, _P, _P], _I32),
            "nd_poisson_create": ([_I32, _I32, ctypes.POINTER(_P)], _I32),
            "nd_poisson_apply": ([_P, _P, _P, _I32, _P], _I32),
            "nd_poisson_solve": ([_P, _D, _P, _P, _I32, _P], _I32),
            "nd_poisson_destroy": ([_P], None),
            "nd_vec_dot": ([_P, _P, _I64, _P, _P], _I32),
            "nd_vec_axpby": ([_D, _P, _D, _P, _I64, _P], _I32),
            "nd_vec_mul": ([_P, _P, _P, _I64, _P], _I32),
            "nd_vec_scale_pos": ([_D, _P, _P, _I64, _P], _I32),
            "nd_profile_launches": ([_P, _P, _I32, ctypes.POINTER(_I32)], _I32),
            "nd_lead_destroy": ([_P], None),
            "nd_sigma_lesser_fermi": ([_P, _I32, _I32, _P, _P, _D, _P, _P, _P, _P], _I32),
            "nd_phonon_const": ([_I32, _I32, _D, _D, _D, _P, _P, _P, _P, _P], _I32),
            "nd_phonon_scba": ([_I32, _I32, _D, _D, _P, _P, _P, _P, _P, _P, _P, _P], _I32),
            "nd_check_factor_inputs": ([_P, _P, _P, _I32], _I32),
            "nd_check_lesser_inputs": ([_P, _P, _P, _P, _P, _I32], _I32),
            "nd_last_error": ([], ctypes.c_char_p),
            "nd_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = L
    return _LIB


def _check(st, name):
    if st != 0:
        raise NDError(st, f"{name}: {lib().nd_last_error().decode()}")


def _ptr(x, keep):
    """Raw pointer of a tensor / array (None -> NULL).  Arrays are kept alive
    in ``keep`` for the duration of the call."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):  # torch tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        keep.append(x)
        return x.data_ptr()
    a = np.ascontiguousarray(x)
    keep.append(a)
    return a.ctypes.data


def require_real(x, name: str):
    """The float64 array that a real Hamiltonian argument (H values, lead
    blocks H00, H01, tau) must be.  Complex values describe a Hermitian H
    that need not be complex symmetric (complex hoppings, e.g. a magnetic
    field); the elimination relies on A = A^T (paper Sec. 3.1), so they are
    rejected with ND_ERR_NOT_SYMMETRIC instead of losing their imaginary part
    in a cast.  Other real numpy dtypes are converted; a torch tensor must
    already be float64.  Returns the array (numpy) or the tensor unchanged."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):  # torch tensor
        if x.is_complex():
            raise NDError(2, f"{name}: complex values; a Hermitian H that is not real symmetric is not supported")
        if str(x.dtype) != "torch.float64":
            raise NDError(1, f"{name}: expected a float64 tensor, got {x.dtype}")
        return x
    a = np.asarray(x)
    if np.iscomplexobj(a):
        raise NDError(2, f"{name}: complex values; a Hermitian H that is not real symmetric is not supported")
    return np.ascontiguousarray(a, dtype=np.float64)


def _need(x, name: str, nbytes: int, complex_ok: bool = True, output: bool = False):
    """Buffer check of the binding (the C ABI sees raw pointers and cannot):
    ``x`` (a numpy array or torch tensor; None passes) holds float64 or, where
    ``complex_ok``, complex128 elements (the ABI's doubles, complex values
    interleaved), at least ``nbytes`` bytes, and, for an output, one
    contiguous block that the library writes in place.  A narrower element
    type would be misread and a short buffer overrun; both are
    ND_ERR_INVALID_ARG here."""
    if x is None:
        return
    if hasattr(x, "data_ptr"):  # torch tensor
        dt, size, contiguous = str(x.dtype).replace("torch.", ""), x.numel() * x.element_size(), x.is_contiguous()
    else:
        a = np.asarray(x)
        dt, size, contiguous = str(a.dtype), a.nbytes, a.flags.c_contiguous and isinstance(x, np.ndarray)
    if not (dt == "float64" or (complex_ok and dt == "complex128")):
        raise NDError(1, f"{name}: elements of type {dt}, expected {'complex128 or ' if complex_ok else ''}float64")
    if size < nbytes:
        raise NDError(1, f"{name}: {size} bytes, the call needs {nbytes}")
    if output and not contiguous:
        raise NDError(1, f"{name}: an output must be one contiguous array")


def _need_i32(x, name: str, count: int, output: bool = False):
    """The int32 counterpart of ``_need``: at least ``count`` int32 elements."""
    if x is None:
        return
    if hasattr(x, "data_ptr"):
        dt, size, contiguous = str(x.dtype).replace("torch.", ""), x.numel(), x.is_contiguous()
    else:
        a = np.asarray(x)
        dt, size, contiguous = str(a.dtype), a.size, a.flags.c_contiguous and isinstance(x, np.ndarray)
    if dt != "int32":
        raise NDError(1, f"{name}: elements of type {dt}, expected int32")
    if size < count:
        raise NDError(1, f"{name}: {size} elements, the call needs {count}")
    if output and not contiguous:
        raise NDError(1, f"{name}: an output must be one contiguous array")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class _Handle:
    _destroy = None

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            getattr(lib(), self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan(_Handle):
    _destroy = "nd_plan_destroy"


class Fact(_Handle):
    _destroy = "nd_fact_destroy"

    def __init__(self, ptr, plan):
        super().__init__(ptr)
        self.plan = plan  # the plan must outlive the workspace
        self.n_e = None  # energies of the last successful nd_factor / nd_autotune (buffer checks)


def _factor_inputs(fact: Fact, name: str, H_values, sigma_r, sigma_ph_r, energies, n_e: int):
    if n_e <= 0:
        return  # the library reports the count
    p = fact.plan
    _need(H_values, f"{name}: H_values", 8 * p.nnz, complex_ok=False)
    _need(sigma_r, f"{name}: sigma_r", 16 * n_e * p.sigma_elems)
    _need(sigma_ph_r, f"{name}: sigma_ph_r", 16 * n_e * p.n)
    _need(energies, f"{name}: energies", 8 * n_e, complex_ok=False)


def _lesser_inputs(fact: Fact, name: str, n_e, sigma_lesser, sigma_greater, ph_lesser, ph_greater):
    p = fact.plan
    _need(sigma_lesser, f"{name}: sigma_lesser", 16 * n_e * p.sigma_elems)
    _need(sigma_greater, f"{name}: sigma_greater", 16 * n_e * p.sigma_elems)
    _need(ph_lesser, f"{name}: ph_lesser", 16 * n_e * p.n)
    _need(ph_greater, f"{name}: ph_greater", 16 * n_e * p.n)


class Lead(_Handle):
    _destroy = "nd_lead_destroy"


class Poisson(_Handle):
    _destroy = "nd_poisson_destroy"


def nd_analyze(n, rowptr, colind, contact_ptr=None, contact_idx=None, coords=None, leaf_size=0,
               split_permille=0, slab=0, delay=0) -> Plan:
    keep = []
    for arr, name in ((rowptr, "rowptr"), (colind, "colind"), (contact_ptr, "contact_ptr"), (contact_idx, "contact_idx")):
        a = np.asarray(arr) if arr is not None else np.zeros(0, np.int32)
        if a.size and (a.dtype.kind not in "iu" or int(a.max()) > np.iinfo(np.int32).max or int(a.min()) < 0):
            # the ABI's indices are int32: a wider value would wrap in the cast
            raise NDError(1, f"nd_analyze: {name} must hold integers in 0..2^31-1")
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    # the library reads these host arrays by the lengths they imply
    if n < 0 or rp.size != n + 1 or ci.size < (int(rp[-1]) if rp.size else 0):
        raise NDError(1, "nd_analyze: rowptr must have n + 1 entries and colind rowptr[n]")
    if contact_ptr is not None:
        cpv = np.asarray(contact_ptr)
        if contact_idx is None or cpv.size < 1 or np.asarray(contact_idx).size < int(cpv[-1]):
            raise NDError(1, "nd_analyze: contact_idx must hold contact_ptr[-1] sites")
    if coords is not None and (np.ndim(coords) != 2 or np.shape(coords)[0] != n):
        raise NDError(1, "nd_analyze: coords must be [n][dim]")
    g = nd_graph()
    g.n = n
    g.rowptr = _ptr(rp, keep)
    g.colind = _ptr(ci, keep)
    if contact_ptr is not None:
        cp = np.ascontiguousarray(contact_ptr, dtype=np.int32)
        cidx = np.ascontiguousarray(contact_idx, dtype=np.int32)
        g.n_contacts = len(cp) - 1
        g.contact_ptr = _ptr(cp, keep)
        g.contact_idx = _ptr(cidx, keep)
    if coords is not None:
        co = np.ascontiguousarray(coords, dtype=np.float64)
        g.coord_dim = co.shape[1]
        g.coords = _ptr(co, keep)
    o = nd_opts()
    o.leaf_size = leaf_size
    o.split_permille = split_permille
    o.slab = slab
    o.delay = delay
    out = _P()
    _check(lib().nd_analyze(ctypes.byref(g), ctypes.byref(o), ctypes.byref(out)), "nd_analyze")
    plan = Plan(out.value)
    plan.n, plan.nnz = int(n), int(rp[-1]) if len(rp) else 0
    plan.sigma_elems = int((np.diff(cp).astype(np.int64) ** 2).sum()) if contact_ptr is not None else 0
    return plan


def nd_plan_query(plan: Plan) -> dict:
    info = nd_plan_info()
    _check(lib().nd_plan_query(plan.ptr, ctypes.byref(info)), "nd_plan_query")
    return {f: getattr(info, f) for f, _ in nd_plan_info._fields_}


def nd_plan_tree(plan: Plan) -> dict:
    info = nd_plan_query(plan)
    nc, n = info["n_clusters"], info["n"]
    arr = {k: np.zeros(nc, dtype=np.int32) for k in ("level", "parent", "n_i", "b_i")}
    arr["cluster_of_site"] = np.zeros(n, dtype=np.int32)
    _check(lib().nd_plan_tree(plan.ptr, arr["level"].ctypes.data, arr["parent"].ctypes.data, arr["n_i"].ctypes.data,
                              arr["b_i"].ctypes.data, arr["cluster_of_site"].ctypes.data), "nd_plan_tree")
    return arr


def nd_plan_cluster_sites(plan: Plan, c: int, n_i: int, b_i: int):
    out = np.zeros(n_i + b_i, dtype=np.int32)
    _check(lib().nd_plan_cluster_sites(plan.ptr, c, out.ctypes.data), "nd_plan_cluster_sites")
    return out[:n_i], out[n_i:]


def nd_fact_create(plan: Plan, max_ne: int, precision: int = ND_PREC_FP64, flags: int = 0) -> Fact:
    if max_ne > 65535:  # energies index the grid's y dimension in every launch
        raise NDError(8, "nd_fact_create: at most 65535 energies per handle")
    out = _P()
    _check(lib().nd_fact_create(plan.ptr, max_ne, precision, flags, ctypes.byref(out)), "nd_fact_create")
    fact = Fact(out.value, plan)
    fact.max_ne = int(max_ne)
    return fact


def nd_factor(fact: Fact, H_values, sigma_r, sigma_ph_r, energies, n_e: int, eta: float, stream=None):
    keep = []
    H_values = require_real(H_values, "nd_factor: H_values")
    _factor_inputs(fact, "nd_factor", H_values, sigma_r, sigma_ph_r, energies, n_e)
    fact.n_e = None
    _check(lib().nd_factor(fact.ptr, _ptr(H_values, keep), _ptr(sigma_r, keep), _ptr(sigma_ph_r, keep),
                           _ptr(energies, keep), n_e, eta, _stream(stream)), "nd_factor")
    fact.n_e = int(n_e)


def nd_diag_green(fact: Fact, sigma_lesser, sigma_greater, ph_lesser, ph_greater, Gr, Gl, Gg, stream=None):
    keep = []
    if fact.n_e is not None:  # without a factorization the library refuses the call
        _lesser_inputs(fact, "nd_diag_green", fact.n_e, sigma_lesser, sigma_greater, ph_lesser, ph_greater)
        for g, name in ((Gr, "Gr"), (Gl, "Gl"), (Gg, "Gg")):
            _need(g, f"nd_diag_green: {name}", 16 * fact.n_e * fact.plan.n, output=True)
    _check(lib().nd_diag_green(fact.ptr, _ptr(sigma_lesser, keep), _ptr(sigma_greater, keep), _ptr(ph_lesser, keep),
                               _ptr(ph_greater, keep), _ptr(Gr, keep), _ptr(Gl, keep), _ptr(Gg, keep),
                               _stream(stream)), "nd_diag_green")


def nd_check_factor_inputs(plan: Plan, H_values, sigma_r, n_e: int):
    """Host-side symmetry check of nd_factor's inputs (host arrays)."""
    keep = []
    H_values = require_real(H_values, "nd_check_factor_inputs: H_values")
    if n_e > 0:
        _need(H_values, "nd_check_factor_inputs: H_values", 8 * plan.nnz, complex_ok=False)
        _need(sigma_r, "nd_check_factor_inputs: sigma_r", 16 * n_e * plan.sigma_elems)
    _check(lib().nd_check_factor_inputs(plan.ptr, _ptr(H_values, keep), _ptr(sigma_r, keep), n_e),
           "nd_check_factor_inputs")


def nd_check_lesser_inputs(plan: Plan, sigma_lesser, sigma_greater, ph_lesser, ph_greater, n_e: int):
    """Host-side skew-Hermiticity check of nd_diag_green's inputs (host arrays)."""
    keep = []
    if n_e > 0:
        for x, name, per in ((sigma_lesser, "sigma_lesser", plan.sigma_elems), (sigma_greater, "sigma_greater",
                             plan.sigma_elems), (ph_lesser, "ph_lesser", plan.n), (ph_greater, "ph_greater", plan.n)):
            _need(x, f"nd_check_lesser_inputs: {name}", 16 * n_e * per)
    _check(lib().nd_check_lesser_inputs(plan.ptr, _ptr(sigma_lesser, keep), _ptr(sigma_greater, keep),
                                        _ptr(ph_lesser, keep), _ptr(ph_greater, keep), n_e), "nd_check_lesser_inputs")


def nd_certificate(fact: Fact, cert, stream=None):
    keep = []
    if fact.n_e is not None:
        _need(cert, "nd_certificate: cert", 64 * fact.n_e, complex_ok=False, output=True)
    _check(lib().nd_certificate(fact.ptr, _ptr(cert, keep), _stream(stream)), "nd_certificate")


def nd_selected_entries(fact: Fact, x, y, count: int, Gr, Gl, Gg, n_missing, stream=None):
    """Selected entries G^r_xy, G^<_xy, G^>_xy of the last solve (device arrays)."""
    keep = []
    if count > 0:
        _need_i32(x, "nd_selected_entries: x", count)
        _need_i32(y, "nd_selected_entries: y", count)
        _need_i32(n_missing, "nd_selected_entries: n_missing", 1, output=True)
        if fact.n_e is not None:
            for g, name in ((Gr, "Gr"), (Gl, "Gl"), (Gg, "Gg")):
                _need(g, f"nd_selected_entries: {name}", 16 * fact.n_e * count, output=True)
    _check(lib().nd_selected_entries(fact.ptr, _ptr(x, keep), _ptr(y, keep), count, _ptr(Gr, keep), _ptr(Gl, keep),
                                     _ptr(Gg, keep), _ptr(n_missing, keep), _stream(stream)), "nd_selected_entries")


def nd_density(Gl, weights, n_e, n, scale, accumulate, out, stream=None):
    keep = []
    if n_e > 0 and n > 0:
        _need(Gl, "nd_density: Gl", 16 * n_e * n)
        _need(weights, "nd_density: weights", 8 * n_e, complex_ok=False)
        _need(out, "nd_density: out", 8 * n, complex_ok=False, output=True)
    _check(lib().nd_density(_ptr(Gl, keep), _ptr(weights, keep), n_e, n, scale, int(accumulate), _ptr(out, keep),
                            _stream(stream)), "nd_density")


def nd_fact_density(fact: Fact, weights, scale, accumulate, out, stream=None):
    """Density epilogue on the handle's last diag G^< (host or device weights / out)."""
    keep = []
    if fact.n_e is not None:
        _need(weights, "nd_fact_density: weights", 8 * fact.n_e, complex_ok=False)
        _need(out, "nd_fact_density: out", 8 * fact.plan.n, complex_ok=False, output=True)
    _check(lib().nd_fact_density(fact.ptr, _ptr(weights, keep), scale, int(accumulate), _ptr(out, keep),
                                 _stream(stream)), "nd_fact_density")


def nd_profile(fact: Fact, enable: bool) -> list:
    """Returns per-kernel-kind stats recorded since the previous call and sets
    the enable state."""
    arr = (nd_kernel_stats * 24)()
    cnt = _I32()
    _check(lib().nd_profile(fact.ptr, int(enable), arr, 24, ctypes.byref(cnt)), "nd_profile")
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "ms": arr[i].ms, "flops": arr[i].flops,
             "bytes": arr[i].bytes} for i in range(cnt.value)]


def nd_invert_c64_noalloc(A, n, batch, n_singular, stream=None):
    """In-place inversion of complex64 matrices without device allocation."""
    keep = []
    if A is not None and 0 < n <= 512 and 0 < batch and batch * n * n <= 1 << 18:  # the library refuses the rest
        if hasattr(A, "data_ptr"):
            dt, size, contiguous = str(A.dtype).replace("torch.", ""), A.numel() * A.element_size(), A.is_contiguous()
        else:
            a = np.asarray(A)
            dt, size, contiguous = str(a.dtype), a.nbytes, a.flags.c_contiguous and isinstance(A, np.ndarray)
        if dt not in ("complex64", "float32"):
            raise NDError(1, f"nd_invert_c64_noalloc: A has elements of type {dt}, expected complex64")
        if size < 8 * batch * n * n or not contiguous:
            raise NDError(1, f"nd_invert_c64_noalloc: A must be one contiguous [batch][n][n] complex64 array")
        _need_i32(n_singular, "nd_invert_c64_noalloc: n_singular", 1, output=True)
    _check(lib().nd_invert_c64_noalloc(_ptr(A, keep), n, batch, _ptr(n_singular, keep), _stream(stream)),
           "nd_invert_c64_noalloc")


def nd_fact_status(fact: Fact) -> int:
    n = _I32()
    st = lib().nd_fact_status(fact.ptr, ctypes.byref(n))
    if st not in (0, 3):
        _check(st, "nd_fact_status")
    return n.value


def nd_fact_set_wait_limit(fact: Fact, polls: int):
    """Polls before a tensor-core wait gives up (0 = default)."""
    _check(lib().nd_fact_set_wait_limit(fact.ptr, int(polls)), "nd_fact_set_wait_limit")


def nd_fact_get_choice(fact: Fact) -> np.ndarray:
    """The kernel of every step (int8, -1 = default rule), flattened over the schedules."""
    n = _I32(0)
    _check(lib().nd_fact_get_choice(fact.ptr, None, 0, ctypes.byref(n)), "nd_fact_get_choice")
    out = np.full(n.value, -1, dtype=np.int8)
    _check(lib().nd_fact_get_choice(fact.ptr, out.ctypes.data_as(_P), n.value, ctypes.byref(n)), "nd_fact_get_choice")
    return out


def nd_fact_set_choice(fact: Fact, choice) -> None:
    """Apply a stored kernel choice (as nd_fact_get_choice returns it)."""
    c = np.ascontiguousarray(np.asarray(choice, dtype=np.int8))
    _check(lib().nd_fact_set_choice(fact.ptr, c.ctypes.data_as(_P), int(c.size)), "nd_fact_set_choice")


def nd_autotune(fact: Fact, H_values, sigma_r, sigma_ph_r, sigma_lesser, sigma_greater, ph_lesser, ph_greater,
                energies, n_e: int, eta: float, reps: int = 1, stream=None) -> dict:
    """Measured kernel choice per GEMM launch (see ndgf.h); returns nd_tune_info as a dict."""
    keep = []
    info = nd_tune_info()
    H_values = require_real(H_values, "nd_autotune: H_values")
    _factor_inputs(fact, "nd_autotune", H_values, sigma_r, sigma_ph_r, energies, n_e)
    if n_e > 0:
        _lesser_inputs(fact, "nd_autotune", n_e, sigma_lesser, sigma_greater, ph_lesser, ph_greater)
    fact.n_e = None
    _check(lib().nd_autotune(fact.ptr, _ptr(H_values, keep), _ptr(sigma_r, keep), _ptr(sigma_ph_r, keep),
                             _ptr(sigma_lesser, keep), _ptr(sigma_greater, keep), _ptr(ph_lesser, keep),
                             _ptr(ph_greater, keep), _ptr(energies, keep), n_e, eta, reps, ctypes.byref(info),
                             _stream(stream)), "nd_autotune")
    fact.n_e = int(n_e)  # the passes leave the factorization of these energies
    return {"ms_default": info.ms_default, "ms_tuned": info.ms_tuned, "gemm_steps": info.gemm_steps,
            "changed": info.changed, "passes": info.passes, "by_kind": list(info.by_kind)}


def nd_density_jvp(fact: Fact, v, t_out, stream=None):
    """Forward terms T[e][j] of the density's derivative along v (see ndgf.h)."""
    keep = []
    if fact.n_e is not None:
        _need(v, "nd_density_jvp: v", 8 * fact.plan.n, complex_ok=False)
        _need(t_out, "nd_density_jvp: t_out", 16 * fact.n_e * fact.plan.n, output=True)
    _check(lib().nd_density_jvp(fact.ptr, _ptr(v, keep), _ptr(t_out, keep), _stream(stream)), "nd_density_jvp")


def nd_poisson_create(nx: int, ny: int) -> Poisson:
    out = _P()
    _check(lib().nd_poisson_create(nx, ny, ctypes.byref(out)), "nd_poisson_create")
    p = Poisson(out.value)
    p.sites = int(nx) * int(ny)
    return p


def nd_poisson_apply(p: Poisson, u, out, batch: int = 1, stream=None):
    keep = []
    if batch > 0 and getattr(p, "sites", None):
        _need(u, "nd_poisson_apply: u", 8 * batch * p.sites, complex_ok=False)
        _need(out, "nd_poisson_apply: out", 8 * batch * p.sites, complex_ok=False, output=True)
    _check(lib().nd_poisson_apply(p.ptr, _ptr(u, keep), _ptr(out, keep), batch, _stream(stream)), "nd_poisson_apply")


def nd_poisson_solve(p: Poisson, rhs, u, batch: int = 1, shift: float = 0.0, stream=None):
    keep = []
    if batch > 0 and getattr(p, "sites", None):
        _need(rhs, "nd_poisson_solve: rhs", 8 * batch * p.sites, complex_ok=False)
        _need(u, "nd_poisson_solve: u", 8 * batch * p.sites, complex_ok=False, output=True)
    _check(lib().nd_poisson_solve(p.ptr, shift, _ptr(rhs, keep), _ptr(u, keep), batch, _stream(stream)),
           "nd_poisson_solve")


def nd_vec_dot(x, y, n: int, out, stream=None):
    keep = []
    if n > 0:
        _need(x, "nd_vec_dot: x", 8 * n, complex_ok=False)
        _need(y, "nd_vec_dot: y", 8 * n, complex_ok=False)
        _need(out, "nd_vec_dot: out", 8, complex_ok=False, output=True)
    _check(lib().nd_vec_dot(_ptr(x, keep), _ptr(y, keep), n, _ptr(out, keep), _stream(stream)), "nd_vec_dot")


def nd_vec_axpby(a: float, x, b: float, y, n: int, stream=None):
    keep = []
    if n > 0:
        _need(x, "nd_vec_axpby: x", 8 * n, complex_ok=False)
        _need(y, "nd_vec_axpby: y", 8 * n, complex_ok=False, output=True)
    _check(lib().nd_vec_axpby(a, _ptr(x, keep), b, _ptr(y, keep), n, _stream(stream)), "nd_vec_axpby")


def nd_vec_mul(d, x, y, n: int, stream=None):
    keep = []
    if n > 0:
        _need(d, "nd_vec_mul: d", 8 * n, complex_ok=False)
        _need(x, "nd_vec_mul: x", 8 * n, complex_ok=False)
        _need(y, "nd_vec_mul: y", 8 * n, complex_ok=False, output=True)
    _check(lib().nd_vec_mul(_ptr(d, keep), _ptr(x, keep), _ptr(y, keep), n, _stream(stream)), "nd_vec_mul")


def nd_vec_scale_pos(a: float, x, y, n: int, stream=None):
    keep = []
    if n > 0:
        _need(x, "nd_vec_scale_pos: x", 8 * n, complex_ok=False)
        _need(y, "nd_vec_scale_pos: y", 8 * n, complex_ok=False, output=True)
    _check(lib().nd_vec_scale_pos(a, _ptr(x, keep), _ptr(y, keep), n, _stream(stream)), "nd_vec_scale_pos")


def nd_lead_create(H00, H01, tau) -> Lead:
    keep = []
    H00 = require_real(H00, "nd_lead_create: H00")
    H01 = require_real(H01, "nd_lead_create: H01")
    tau = require_real(tau, "nd_lead_create: tau")
    m = H00.shape[0]
    out = _P()
    _check(lib().nd_lead_create(m, tau.shape[0], _ptr(H00, keep), _ptr(H01, keep),
                                _ptr(tau, keep), ctypes.byref(out)), "nd_lead_create")
    lead = Lead(out.value)
    lead.m_c = int(tau.shape[0])
    return lead


def nd_lead_sigma(lead: Lead, energies, n_e: int, eta: float, sigma_out, stride: int, offset: int, stream=None):
    keep = []
    m_c = getattr(lead, "m_c", None)
    if n_e > 0 and m_c is not None and stride >= 0 and offset >= 0:
        _need(energies, "nd_lead_sigma: energies", 8 * n_e, complex_ok=False)
        _need(sigma_out, "nd_lead_sigma: sigma_out", 16 * ((n_e - 1) * stride + offset + m_c * m_c), output=True)
    _check(lib().nd_lead_sigma(lead.ptr, _ptr(energies, keep), n_e, eta, _ptr(sigma_out, keep), stride, offset,
                               _stream(stream)), "nd_lead_sigma")


class nd_launch_stats(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("count", ctypes.c_int32), ("max_dim", ctypes.c_int32),
                ("n_e", ctypes.c_int32), ("ms", ctypes.c_double), ("flops", ctypes.c_double)]


def nd_profile_launches(fact: Fact):
    """Per-launch records of the profiler (see nd_profile), in launch order."""
    n = _I32()
    _check(lib().nd_profile_launches(fact.ptr, None, 0, ctypes.byref(n)), "nd_profile_launches")
    arr = (nd_launch_stats * max(1, n.value))()
    _check(lib().nd_profile_launches(fact.ptr, arr, n.value, ctypes.byref(n)), "nd_profile_launches")
    return [dict(kind=r.kind, count=r.count, max_dim=r.max_dim, n_e=r.n_e, ms=r.ms, flops=r.flops)
            for r in arr[:n.value]]


def nd_density_gradient(fact: Fact, c, t_out, stream=None):
    """t_out[e][k] = sum_ab Sigma^<_ab conj(U_kb) conj(Z_ka) of the last step (see ndgf.h)."""
    keep = []
    if fact.n_e is not None:
        _need(c, "nd_density_gradient: c", 8 * fact.plan.n, complex_ok=False)
        _need(t_out, "nd_density_gradient: t_out", 16 * fact.n_e * fact.plan.n, output=True)
    _check(lib().nd_density_gradient(fact.ptr, _ptr(c, keep), _ptr(t_out, keep), _stream(stream)),
           "nd_density_gradient")


def nd_contact_current(fact: Fact, contact: int, current, current_im=None, stream=None):
    keep = []
    if fact.n_e is not None:
        _need(current, "nd_contact_current: current", 8 * fact.n_e, complex_ok=False, output=True)
        _need(current_im, "nd_contact_current: current_im", 8 * fact.n_e, complex_ok=False, output=True)
    _check(lib().nd_contact_current(fact.ptr, contact, _ptr(current, keep),
                                    _ptr(current_im, keep) if current_im is not None else None, _stream(stream)),
           "nd_contact_current")


def nd_lead_status(lead: Lead):
    """(n_unconverged, n_singular) of the decimation since the previous call."""
    a, b = _I32(), _I32()
    st = lib().nd_lead_status(lead.ptr, ctypes.byref(a), ctypes.byref(b))
    if st not in (0, 3):
        _check(st, "nd_lead_status")
    return a.value, b.value


def nd_sigma_lesser_fermi(sigma_r, n_e, m_c, mu, kT, energies, sigma_lesser, sigma_greater, stream=None):
    keep = []
    mc = np.ascontiguousarray(m_c, dtype=np.int32)
    muv = np.ascontiguousarray(mu, dtype=np.float64)
    if muv.size < mc.size:
        raise NDError(1, "nd_sigma_lesser_fermi: one Fermi level per contact")
    if n_e > 0:
        elems = int((mc.astype(np.int64) ** 2).sum())
        _need(sigma_r, "nd_sigma_lesser_fermi: sigma_r", 16 * n_e * elems)
        _need(energies, "nd_sigma_lesser_fermi: energies", 8 * n_e, complex_ok=False)
        _need(sigma_lesser, "nd_sigma_lesser_fermi: sigma_lesser", 16 * n_e * elems, output=True)
        _need(sigma_greater, "nd_sigma_lesser_fermi: sigma_greater", 16 * n_e * elems, output=True)
    _check(lib().nd_sigma_lesser_fermi(_ptr(sigma_r, keep), n_e, len(mc), _ptr(mc, keep), _ptr(muv, keep), kT,
                                       _ptr(energies, keep), _ptr(sigma_lesser, keep), _ptr(sigma_greater, keep),
                                       _stream(stream)), "nd_sigma_lesser_fermi")


def nd_phonon_const(n, n_e, gamma, mu, kT, energies, ph_r, ph_lesser, ph_greater, stream=None):
    keep = []
    if n > 0 and n_e > 0:
        _need(energies, "nd_phonon_const: energies", 8 * n_e, complex_ok=False)
        for x, name in ((ph_r, "ph_r"), (ph_lesser, "ph_lesser"), (ph_greater, "ph_greater")):
            _need(x, f"nd_phonon_const: {name}", 16 * n_e * n, output=True)
    _check(lib().nd_phonon_const(n, n_e, gamma, mu, kT, _ptr(energies, keep), _ptr(ph_r, keep),
                                 _ptr(ph_lesser, keep), _ptr(ph_greater, keep), _stream(stream)), "nd_phonon_const")


def nd_phonon_scba(n, n_e, D, mix, Gr, Gl, Gg, ph_r, ph_lesser, ph_greater, stats, stream=None):
    """Self-consistent Born update of the elastic local phonon self-energy (see ndgf.h)."""
    keep = []
    if n > 0 and n_e > 0:
        for x, name in ((Gr, "Gr"), (Gl, "Gl"), (Gg, "Gg")):
            _need(x, f"nd_phonon_scba: {name}", 16 * n_e * n)
        for x, name in ((ph_r, "ph_r"), (ph_lesser, "ph_lesser"), (ph_greater, "ph_greater")):
            _need(x, f"nd_phonon_scba: {name}", 16 * n_e * n, output=True)
        _need(stats, "nd_phonon_scba: stats", 16, complex_ok=False, output=True)
    _check(lib().nd_phonon_scba(n, n_e, D, mix, _ptr(Gr, keep), _ptr(Gl, keep), _ptr(Gg, keep), _ptr(ph_r, keep),
                                _ptr(ph_lesser, keep), _ptr(ph_greater, keep), _ptr(stats, keep), _stream(stream)),
           "nd_phonon_scba")


def nd_version() -> str:
    return lib().nd_version().decode()
