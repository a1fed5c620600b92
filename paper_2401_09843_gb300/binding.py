"""Thin ctypes binding of the C ABI in include/ns3d.h.

Argument marshalling only: every step of the solver runs in libns3d.so.
Device buffers are PyTorch CUDA tensors (complex64 for NS3D_F32, complex128
for NS3D_F64) in the D1 layout [3][N][N][N/2+1]; the plan's stream is the
PyTorch stream current when the plan is created.  There is no CPU fallback:
``load`` raises when the library is missing or a call fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libns3d.so")

NS3D_F32, NS3D_F64 = 0, 1
STATUS = {0: "NS3D_OK", 1: "NS3D_ERR_INVALID_ARG", 2: "NS3D_ERR_OUT_OF_MEMORY",
          3: "NS3D_ERR_CUDA", 4: "NS3D_ERR_NONFINITE", 5: "NS3D_ERR_UNSTABLE_DT",
          6: "NS3D_ERR_TIMEOUT", 7: "NS3D_ERR_NOT_SUPPORTED"}

# every symbol include/ns3d.h declares
SYMBOLS = ["ns3d_params_default", "ns3d_plan_create", "ns3d_plan_destroy", "ns3d_plan_info",
           "ns3d_set_initial", "ns3d_get_state", "ns3d_step", "ns3d_synchronize",
           "ns3d_eval_rhs", "ns3d_adjoint_step", "ns3d_grad_band_energy",
           "ns3d_ensemble_stats", "ns3d_status_string", "ns3d_step_timed",
           "ns3d_eval_rhs_noalloc", "ns3d_test_stall_staging", "ns3d_get_clock",
           "ns3d_set_clock", "ns3d_test_poison_workspaces", "ns3d_vorticity_magnitude",
           "ns3d_physical_field", "ns3d_band_energy", "ns3d_mesh_refinement",
           "ns3d_project"]


class Ns3dError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("nu", ctypes.c_double), ("s", ctypes.c_double),
                ("theta", ctypes.c_double), ("eps0", ctypes.c_double),
                ("mN_coef", ctypes.c_double), ("q_form", ctypes.c_int), ("n_pad", ctypes.c_int),
                ("nonlinear_form", ctypes.c_int), ("cfl", ctypes.c_double),
                ("dt_fixed", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("second", ctypes.c_void_p), ("var", ctypes.c_void_p),
                ("spectrum", ctypes.c_void_p), ("spectrum_se", ctypes.c_void_p),
                ("s2", ctypes.c_void_p), ("s2_se", ctypes.c_void_p),
                ("energy", ctypes.c_double), ("energy_se", ctypes.c_double),
                ("members", ctypes.c_int),
                ("enstrophy_spectrum", ctypes.c_void_p), ("enstrophy_spectrum_se", ctypes.c_void_p),
                ("enstrophy", ctypes.c_double), ("enstrophy_se", ctypes.c_double),
                ("dissipation", ctypes.c_double), ("dissipation_se", ctypes.c_double),
                ("s2_ball", ctypes.c_void_p), ("s2_ball_se", ctypes.c_void_p)]


class Refinement(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_double * 3), ("mean_err", ctypes.c_double * 3),
                ("var_err", ctypes.c_double * 3), ("sample_err", ctypes.c_double * 3),
                ("mc_se", ctypes.c_double * 3), ("coarse_members", ctypes.c_int),
                ("fine_members", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libns3d.so (once) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2401_09843_gb300.build")
    lib = ctypes.CDLL(path)
    vp, ip, i, d, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "ns3d_params_default": (None, [ctypes.POINTER(Params)]),
        "ns3d_plan_create": (i, [ctypes.POINTER(vp), ip, i, i, ctypes.POINTER(Params), vp, sz]),
        "ns3d_plan_destroy": (i, [vp]),
        "ns3d_plan_info": (i, [vp, i, ip, ip, ctypes.POINTER(sz), ip]),
        "ns3d_set_initial": (i, [vp, i, vp, i]),
        "ns3d_get_state": (i, [vp, i, vp, i, ctypes.POINTER(d)]),
        "ns3d_step": (i, [vp, i, d]),
        "ns3d_synchronize": (i, [vp]),
        "ns3d_eval_rhs": (i, [vp, i, vp, vp, i]),
        "ns3d_adjoint_step": (i, [vp, i, vp, vp, vp, i]),
        "ns3d_grad_band_energy": (i, [vp, i, d, d, i, i, vp, i]),
        "ns3d_ensemble_stats": (i, [vp, i, ctypes.POINTER(Stats)]),
        "ns3d_status_string": (ctypes.c_char_p, [i]),
        "ns3d_step_timed": (i, [vp, i, d, ctypes.POINTER(d), ip]),
        "ns3d_eval_rhs_noalloc": (i, [i, i, ctypes.POINTER(Params), vp, vp, vp]),
        "ns3d_test_stall_staging": (i, [vp, i]),
        "ns3d_get_clock": (i, [vp, i, ctypes.POINTER(d), ip]),
        "ns3d_set_clock": (i, [vp, i, d, i]),
        "ns3d_test_poison_workspaces": (i, [vp]),
        "ns3d_vorticity_magnitude": (i, [vp, i, vp, i]),
        "ns3d_physical_field": (i, [vp, i, vp, i]),
        "ns3d_band_energy": (i, [vp, i, d, d, ctypes.POINTER(d)]),
        "ns3d_mesh_refinement": (i, [vp, i, i, ctypes.POINTER(Refinement)]),
        "ns3d_project": (i, [vp, i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code: int, what: str):
    if code != 0:
        raise Ns3dError(code, what)


def default_params(**kw) -> Params:
    p = Params()
    load().ns3d_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def eval_rhs_noalloc(uhat, dtype: int = NS3D_F64, params: Params | None = None, stream=None):
    """R(u_hat) through ns3d_eval_rhs_noalloc (no plan, no device allocation in
    the library; N <= 32).  uhat: CUDA tensor in D1 layout of the dtype."""
    import torch
    lib = load()
    p = params if params is not None else default_params()
    s = stream if stream is not None else torch.cuda.current_stream()
    out = torch.empty_like(uhat)
    _check(lib.ns3d_eval_rhs_noalloc(int(uhat.shape[-2]), dtype, ctypes.byref(p),
                                     ctypes.c_void_p(uhat.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(s.cuda_stream)), "ns3d_eval_rhs_noalloc")
    return out


class Plan:
    """An ensemble of members (resolutions N_per_member) advanced on one GPU."""

    def __init__(self, N_per_member, dtype: int = NS3D_F32, params: Params | None = None,
                 stream=None, workspace_limit: int = 0, **param_kw):
        import torch
        self.lib = load()
        self.torch = torch
        self.dtype = dtype
        self.cdtype = torch.complex64 if dtype == NS3D_F32 else torch.complex128
        self.N = [int(n) for n in N_per_member]
        p = params if params is not None else default_params()
        for k, v in param_kw.items():
            setattr(p, k, v)
        self.params = p
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (ctypes.c_int * len(self.N))(*self.N)
        h = ctypes.c_void_p()
        _check(self.lib.ns3d_plan_create(ctypes.byref(h), arr, len(self.N), dtype, ctypes.byref(p),
                                         ctypes.c_void_p(self.stream.cuda_stream), workspace_limit),
               "ns3d_plan_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            _check(self.lib.ns3d_plan_destroy(self.h), "ns3d_plan_destroy")
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def _d1_shape(self, member):
        n = self.N[member]
        return (3, n, n, n // 2 + 1)

    def _as_dev(self, x, member):
        t = self.torch
        if isinstance(x, np.ndarray):
            x = t.from_numpy(np.ascontiguousarray(x))
        x = x.to(device="cuda", dtype=self.cdtype).contiguous()
        if tuple(x.shape) != self._d1_shape(member):
            raise ValueError(f"expected shape {self._d1_shape(member)}, got {tuple(x.shape)}")
        return x

    def info(self, member: int = 0):
        N, P, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        b = ctypes.c_size_t()
        _check(self.lib.ns3d_plan_info(self.h, member, ctypes.byref(N), ctypes.byref(P), ctypes.byref(b),
                                       ctypes.byref(nl)), "ns3d_plan_info")
        return dict(N=N.value, P=P.value, device_bytes=b.value, launches_per_step=nl.value)

    # ------------------------------------------------------------ API
    def set_initial(self, member: int, uhat):
        x = self._as_dev(uhat, member)
        _check(self.lib.ns3d_set_initial(self.h, member, ctypes.c_void_p(x.data_ptr()), 1),
               "ns3d_set_initial")
        self._keep = x          # stream-ordered: keep alive until the next call

    def set_initial_host(self, member: int, uhat: np.ndarray):
        npd = np.complex64 if self.dtype == NS3D_F32 else np.complex128
        x = np.ascontiguousarray(uhat, dtype=npd)
        if x.shape != self._d1_shape(member):
            raise ValueError("bad shape")
        _check(self.lib.ns3d_set_initial(self.h, member, x.ctypes.data_as(ctypes.c_void_p), 0),
               "ns3d_set_initial")

    def get_state(self, member: int, with_time: bool = False):
        out = self.torch.empty(self._d1_shape(member), dtype=self.cdtype, device="cuda")
        t = ctypes.c_double()
        _check(self.lib.ns3d_get_state(self.h, member, ctypes.c_void_p(out.data_ptr()), 1, ctypes.byref(t)),
               "ns3d_get_state")
        return (out, t.value) if with_time else out

    def get_state_host(self, member: int, out: np.ndarray | None = None):
        npd = np.complex64 if self.dtype == NS3D_F32 else np.complex128
        if out is None:
            out = np.empty(self._d1_shape(member), dtype=npd)
        t = ctypes.c_double()
        _check(self.lib.ns3d_get_state(self.h, member, out.ctypes.data_as(ctypes.c_void_p), 0, ctypes.byref(t)),
               "ns3d_get_state")
        return out, t.value

    def test_poison_workspaces(self):
        """Test hook: NaN-fill the workspaces and stage buffer (see ns3d.h)."""
        _check(self.lib.ns3d_test_poison_workspaces(self.h), "ns3d_test_poison_workspaces")

    def clock(self, member: int):
        """(t, completed steps) of a member; synchronises."""
        t = ctypes.c_double()
        n = ctypes.c_int()
        _check(self.lib.ns3d_get_clock(self.h, member, ctypes.byref(t), ctypes.byref(n)), "ns3d_get_clock")
        return t.value, n.value

    def set_clock(self, member: int, t: float, nsteps: int):
        _check(self.lib.ns3d_set_clock(self.h, member, ctypes.c_double(t), int(nsteps)), "ns3d_set_clock")

    def step(self, nsteps: int = 1, t_end: float = 0.0):
        _check(self.lib.ns3d_step(self.h, int(nsteps), float(t_end)), "ns3d_step")

    def step_timed(self, nsteps: int = 1, t_end: float = 0.0):
        """Eager steps with CUDA events around each kernel kind; returns
        (milliseconds per kind, launches per kind), kinds = inverse x,
        inverse y, z pass, forward y, forward x, spectral."""
        ms = (ctypes.c_double * 6)()
        nl = (ctypes.c_int * 6)()
        _check(self.lib.ns3d_step_timed(self.h, int(nsteps), float(t_end), ms, nl), "ns3d_step_timed")
        return list(ms), list(nl)

    def synchronize(self):
        _check(self.lib.ns3d_synchronize(self.h), "ns3d_synchronize")

    def test_stall_staging(self, on: bool):
        """Test hook: the fused x pass's first staged tile never completes,
        so its bounded waits time out (the next status read reports
        TIMEOUT).  For tests of the failure path only."""
        _check(self.lib.ns3d_test_stall_staging(self.h, int(bool(on))), "ns3d_test_stall_staging")

    def eval_rhs(self, member: int, uhat):
        x = self._as_dev(uhat, member)
        out = self.torch.empty_like(x)
        _check(self.lib.ns3d_eval_rhs(self.h, member, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), 1), "ns3d_eval_rhs")
        return out

    def adjoint_step(self, member: int, lam_np1, uhat_n):
        l1 = self._as_dev(lam_np1, member)
        u = self._as_dev(uhat_n, member)
        out = self.torch.empty_like(l1)
        _check(self.lib.ns3d_adjoint_step(self.h, member, ctypes.c_void_p(l1.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1),
               "ns3d_adjoint_step")
        return out

    def grad_band_energy(self, member: int, k_lo: float, k_hi: float, nsteps: int,
                         checkpoint_every: int = 0):
        out = self.torch.empty(self._d1_shape(member), dtype=self.cdtype, device="cuda")
        _check(self.lib.ns3d_grad_band_energy(self.h, member, float(k_lo), float(k_hi), int(nsteps),
                                              int(checkpoint_every), ctypes.c_void_p(out.data_ptr()), 1),
               "ns3d_grad_band_energy")
        return out

    def project(self, member: int):
        """Leray-project the member's state in place (ns3d_project)."""
        _check(self.lib.ns3d_project(self.h, member), "ns3d_project")

    def band_energy(self, member: int, k_lo: float, k_hi: float) -> float:
        """J = 1/2 sum_{k_lo <= |k| < k_hi} |u_hat_k|^2 of the member's state."""
        J = ctypes.c_double(0.0)
        _check(self.lib.ns3d_band_energy(self.h, member, float(k_lo), float(k_hi), ctypes.byref(J)),
               "ns3d_band_energy")
        return J.value

    def mesh_refinement(self, coarse_N: int, fine_N: int) -> dict:
        """Section 6.1 measures between the levels coarse_N and fine_N, per
        velocity component (see ns3d_mesh_refinement)."""
        r = Refinement()
        _check(self.lib.ns3d_mesh_refinement(self.h, int(coarse_N), int(fine_N), ctypes.byref(r)),
               "ns3d_mesh_refinement")
        out = {k: [float(x) for x in getattr(r, k)]
               for k in ("w1", "mean_err", "var_err", "sample_err", "mc_se")}
        out["coarse_members"], out["fine_members"] = r.coarse_members, r.fine_members
        return out

    def ensemble_stats(self, level_N: int, fields: bool = True, ball: bool = True):
        N = int(level_N)
        res = {}
        arrays = {}
        if fields:
            arrays["mean"] = np.zeros((3, N, N, N))
            arrays["second"] = np.zeros((6, N, N, N))
            arrays["var"] = np.zeros((3, N, N, N))
        arrays["spectrum"] = np.zeros(N)
        arrays["spectrum_se"] = np.zeros(N)
        arrays["s2"] = np.zeros(N // 2)
        arrays["s2_se"] = np.zeros(N // 2)
        arrays["enstrophy_spectrum"] = np.zeros(N)
        arrays["enstrophy_spectrum_se"] = np.zeros(N)
        if ball:
            arrays["s2_ball"] = np.zeros(N // 2)
            arrays["s2_ball_se"] = np.zeros(N // 2)
        st = Stats()
        for k, v in arrays.items():
            setattr(st, k, v.ctypes.data_as(ctypes.c_void_p))
        _check(self.lib.ns3d_ensemble_stats(self.h, N, ctypes.byref(st)), "ns3d_ensemble_stats")
        res.update(arrays)
        for k in ("energy", "energy_se", "enstrophy", "enstrophy_se", "dissipation", "dissipation_se"):
            res[k] = getattr(st, k)
        res["members"] = st.members
        return res

    def physical_field(self, member: int):
        """u(x) on the member's N^3 grid: a CUDA tensor [3][N][N][N]."""
        n = self.N[member]
        rdt = self.torch.float32 if self.dtype == NS3D_F32 else self.torch.float64
        out = self.torch.empty((3, n, n, n), dtype=rdt, device="cuda")
        _check(self.lib.ns3d_physical_field(self.h, member, ctypes.c_void_p(out.data_ptr()), 1),
               "ns3d_physical_field")
        return out

    def vorticity_magnitude(self, member: int):
        """|omega(x)| on the member's N^3 grid: a CUDA tensor [N][N][N]."""
        n = self.N[member]
        rdt = self.torch.float32 if self.dtype == NS3D_F32 else self.torch.float64
        out = self.torch.empty((n, n, n), dtype=rdt, device="cuda")
        _check(self.lib.ns3d_vorticity_magnitude(self.h, member, ctypes.c_void_p(out.data_ptr()), 1),
               "ns3d_vorticity_magnitude")
        return out
