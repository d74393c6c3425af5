"""Thin ctypes binding of libgeomhd.so (C ABI: include/geomhd.h).

Argument marshalling only: every step of the method runs in the CUDA library.
If the library is missing, importing this module raises; there is no fallback.
Host arrays are numpy float64 (C order); device arrays are torch CUDA tensors
(float64, contiguous), passed by data pointer.
"""
import ctypes
import os

import numpy as np

from . import _build

GEO_OK = 0
GEO_ERR_ARG = -1
GEO_ERR_OOM = -2
GEO_ERR_CUDA = -3
GEO_ERR_NONPHYSICAL = -4
GEO_ERR_STATE = -6
GEO_FP64 = 0
GEO_FP32_BULK = 1
N_STAGES = 7
STAGES = ("weno", "bperp", "ader", "face_flux", "edge_emf", "update_u", "update_phi")

if not os.path.exists(_build.LIB):
    raise ImportError("libgeomhd.so is not built: run __graft_entry__.build() (or "
                      "python -m paper_1905_02504_gb300._build) on this machine first")

_lib = ctypes.CDLL(_build.LIB)
_d = ctypes.c_double
_i64 = ctypes.c_int64
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p
_h = ctypes.c_void_p

_SIGS = {
    "geo_mesh_create": [ctypes.c_int, ctypes.c_int, _d, _d, ctypes.c_int, ctypes.c_int, _vp,
                        ctypes.POINTER(_h)],
    "geo_mesh_destroy": [_h],
    "geo_mesh_sizes": [_h, _pi64, _pi64, _pi64],
    "geo_set_gamma": [_h, _d],
    "geo_set_positivity": [_h, ctypes.c_int],
    "geo_set_predictor": [_h, ctypes.c_int],
    "geo_set_riemann": [_h, ctypes.c_int],
    "geo_check_state": [_h, ctypes.POINTER(ctypes.c_int)],
    "geo_zone_cubature": [_h, ctypes.c_int, _vp, _vp],
    "geo_edge_quadrature": [_h, ctypes.c_int, _vp, _vp],
    "geo_radial_face_quadrature": [_h, ctypes.c_int, _vp, _vp],
    "geo_phi_from_edge_circulation": [_h, _vp, _vp],
    "geo_zone_geometry": [_h, _vp, _vp],
    "geo_face_geometry": [_h, _vp, _vp],
    "geo_state_upload": [_h, _vp, _vp, ctypes.c_int],
    "geo_state_download": [_h, _vp, _vp, ctypes.c_int],
    "geo_cfl_dt": [_h, _d, _pd],
    "geo_step": [_h, _d],
    "geo_divB_max": [_h, _pd, _pd],
    "geo_set_stage_timing": [_h, ctypes.c_int],
    "geo_get_stage_timing": [_h, _vp, _vp],
    "geo_stage_flops": [_h, _vp, _vp],
    "geo_probe_fma_peak": [ctypes.c_int, _vp, _pd],
    "geo_probe_contraction": [_h, ctypes.c_int, _i64, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_float)],
    "geo_prism_predictor": [ctypes.c_int, _i64, _vp, _vp, _d, _d, _vp, _vp],
    "geo_prism_nodes": [ctypes.c_int, _vp, _i64],
    "geo_prism_derivatives": [ctypes.c_int, _vp, _i64],
    "geo_time_matrix": [ctypes.c_int, _vp, _i64],
    "geo_host_geometry": [ctypes.c_int, ctypes.c_int, _d, _d, ctypes.c_int, _i64, _i64, _vp, _vp, _vp, _vp],
    "geo_debug_buffer": [_h, ctypes.c_int, _vp, _i64],
    "geo_debug_set_buffer": [_h, ctypes.c_int, _vp, _i64],
    "geo_debug_run_stage": [_h, ctypes.c_int, _d],
    "geo_debug_stage_vjp": [_h, ctypes.c_int, _d, _vp, _vp, _vp, _i64, _vp, _i64],
    "geo_cfl_dt_noalloc": [_h, _vp, _d, _vp],
    "geo_step_adjoint": [_h, _d, _vp, _vp, _vp, _vp, _vp, _vp],
    "geo_outer_Br2": [_h, _vp, _pd, _vp],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.geo_last_error.argtypes = []
_lib.geo_last_error.restype = ctypes.c_char_p

EXPORTED = tuple(_SIGS) + ("geo_last_error",)


class GeoError(RuntimeError):
    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


def _check(rc, what):
    if rc != GEO_OK:
        raise GeoError("%s failed (%d): %s" % (what, rc, _lib.geo_last_error().decode()), rc)


def _ptr(a):
    """Data pointer of a numpy array or a torch tensor (must be float64 contiguous)."""
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(_vp)
    assert a.dtype.is_floating_point and a.element_size() == 8 and a.is_contiguous()
    return _vp(a.data_ptr())


def _is_device(a):
    return not isinstance(a, np.ndarray) and a.is_cuda


# ---------------------------------------------------------------- C names
def geo_mesh_create(subdiv, nr, r_in, r_out, order, prec=GEO_FP64, stream=0):
    h = _h()
    _check(_lib.geo_mesh_create(subdiv, nr, r_in, r_out, order, prec, _vp(stream), ctypes.byref(h)),
           "geo_mesh_create")
    return h


def geo_mesh_destroy(h):
    _check(_lib.geo_mesh_destroy(h), "geo_mesh_destroy")


def geo_mesh_sizes(h):
    z, f, e = _i64(), _i64(), _i64()
    _check(_lib.geo_mesh_sizes(h, ctypes.byref(z), ctypes.byref(f), ctypes.byref(e)), "geo_mesh_sizes")
    return z.value, f.value, e.value


def geo_set_gamma(h, gamma):
    _check(_lib.geo_set_gamma(h, gamma), "geo_set_gamma")


def geo_set_positivity(h, enable):
    _check(_lib.geo_set_positivity(h, int(enable)), "geo_set_positivity")


GEO_PRED_ZONE_THREAD = 0
GEO_PRED_NODE_TEAM = 1
GEO_PRED_VAR_TEAM = 2
GEO_RIEMANN_HLL = 0
GEO_RIEMANN_HLLD = 1


def geo_set_riemann(h, solver):
    _check(_lib.geo_set_riemann(h, int(solver)), "geo_set_riemann")


def geo_set_predictor(h, schedule):
    _check(_lib.geo_set_predictor(h, int(schedule)), "geo_set_predictor")


def geo_check_state(h):
    """Physical-state flags raised since the last upload or check (cleared);
    raises GeoError with GEO_ERR_NONPHYSICAL when any is set."""
    flags = ctypes.c_int(0)
    _check(_lib.geo_check_state(h, ctypes.byref(flags)), "geo_check_state")
    return flags.value


def geo_zone_cubature(h, nq):
    Z, _, _ = geo_mesh_sizes(h)
    pts = np.empty((Z, nq ** 3, 3))
    w = np.empty((Z, nq ** 3))
    _check(_lib.geo_zone_cubature(h, nq, _ptr(pts), _ptr(w)), "geo_zone_cubature")
    return pts, w


def geo_edge_quadrature(h, nq):
    _, _, E = geo_mesh_sizes(h)
    pts = np.empty((E, nq, 3))
    tw = np.empty((E, nq, 3))
    _check(_lib.geo_edge_quadrature(h, nq, _ptr(pts), _ptr(tw)), "geo_edge_quadrature")
    return pts, tw


def geo_radial_face_quadrature(h, nq, nrad):
    """nrad = ncol (nr + 1), the number of radial faces of the mesh."""
    pts = np.empty((nrad, nq * nq, 3))
    wn = np.empty((nrad, nq * nq, 3))
    _check(_lib.geo_radial_face_quadrature(h, nq, _ptr(pts), _ptr(wn)), "geo_radial_face_quadrature")
    return pts, wn


def geo_phi_from_edge_circulation(h, circ):
    _, F, _ = geo_mesh_sizes(h)
    circ = np.ascontiguousarray(circ, dtype=np.float64)
    phi = np.empty(F)
    _check(_lib.geo_phi_from_edge_circulation(h, _ptr(circ), _ptr(phi)), "geo_phi_from_edge_circulation")
    return phi


def geo_face_geometry(h):
    _, F, _ = geo_mesh_sizes(h)
    area = np.empty(F)
    nrm = np.empty((F, 3))
    _check(_lib.geo_face_geometry(h, _ptr(area), _ptr(nrm)), "geo_face_geometry")
    return area, nrm


def geo_zone_geometry(h):
    Z, _, _ = geo_mesh_sizes(h)
    xc = np.empty((Z, 3))
    vol = np.empty(Z)
    _check(_lib.geo_zone_geometry(h, _ptr(xc), _ptr(vol)), "geo_zone_geometry")
    return xc, vol


def geo_state_upload(h, U, phi):
    """U: (8, Z) float64, phi: (F,) float64; numpy (host) or torch CUDA tensors."""
    dev = _is_device(U)
    assert dev == _is_device(phi)
    _check(_lib.geo_state_upload(h, _ptr(U), _ptr(phi), int(dev)), "geo_state_upload")


def geo_state_download(h, U, phi):
    dev = _is_device(U)
    assert dev == _is_device(phi)
    _check(_lib.geo_state_download(h, _ptr(U), _ptr(phi), int(dev)), "geo_state_download")


def geo_cfl_dt(h, cfl):
    dt = _d()
    _check(_lib.geo_cfl_dt(h, cfl, ctypes.byref(dt)), "geo_cfl_dt")
    return dt.value


def geo_step(h, dt):
    _check(_lib.geo_step(h, dt), "geo_step")


def geo_divB_max(h):
    a, r = _d(), _d()
    _check(_lib.geo_divB_max(h, ctypes.byref(a), ctypes.byref(r)), "geo_divB_max")
    return a.value, r.value


def geo_set_stage_timing(h, enable):
    _check(_lib.geo_set_stage_timing(h, int(enable)), "geo_set_stage_timing")


def geo_get_stage_timing(h):
    ms = np.zeros(N_STAGES)
    cnt = np.zeros(N_STAGES, dtype=np.int64)
    _check(_lib.geo_get_stage_timing(h, _ptr(ms), cnt.ctypes.data_as(_vp)), "geo_get_stage_timing")
    return ms, cnt


def geo_stage_flops(h):
    fl = np.zeros(N_STAGES)
    units = np.zeros(N_STAGES, dtype=np.int64)
    _check(_lib.geo_stage_flops(h, _ptr(fl), units.ctypes.data_as(_vp)), "geo_stage_flops")
    return fl, units


def geo_probe_fma_peak(prec=GEO_FP64, stream=0):
    v = _d()
    _check(_lib.geo_probe_fma_peak(prec, _vp(stream), ctypes.byref(v)), "geo_probe_fma_peak")
    return v.value


def geo_prism_nodes(order):
    """Reference coordinates of the order's prism nodes, (N, 3)."""
    n = {2: 6, 3: 15, 4: 26}[order]
    out = np.empty((n, 3))
    _check(_lib.geo_prism_nodes(order, _ptr(out), out.size), "geo_prism_nodes")
    return out


def geo_host_geometry(subdiv, nr, r_in, r_out, order, zones, faces):
    """(centroid (Z, 3), volume (Z,), area (F,), normal (F, 3)) from the host tables."""
    xc, vol = np.empty((zones, 3)), np.empty(zones)
    area, nrm = np.empty(faces), np.empty((faces, 3))
    _check(_lib.geo_host_geometry(subdiv, nr, r_in, r_out, order, zones, faces, _ptr(xc), _ptr(vol), _ptr(area),
                                  _ptr(nrm)), "geo_host_geometry")
    return xc, vol, area, nrm


def geo_time_matrix(order):
    """The predictor's R, (M, M) with M = order."""
    out = np.empty((order, order))
    _check(_lib.geo_time_matrix(order, _ptr(out), out.size), "geo_time_matrix")
    return out


def geo_prism_derivatives(order):
    """The prism's D^alpha, (3, N, N)."""
    n = {2: 6, 3: 15, 4: 26}[order]
    out = np.empty((3, n, n))
    _check(_lib.geo_prism_derivatives(order, _ptr(out), out.size), "geo_prism_derivatives")
    return out


def geo_prism_predictor(order, X, U, dt, gamma, Uh, stream=0):
    """X [3][N][Z], U [8][N][Z], Uh [M][8][N][Z]: float64 CUDA tensors."""
    for t in (X, U, Uh):
        assert _is_device(t)
    Z = X.shape[-1]
    _check(_lib.geo_prism_predictor(order, Z, _ptr(X), _ptr(U), dt, gamma, _ptr(Uh), _vp(stream)),
           "geo_prism_predictor")


def geo_probe_contraction(h, tensor, zones, reps, out):
    """out: float32 CUDA tensor of zones x 8 x N elements; returns the launch's ms."""
    ms = ctypes.c_float()
    _check(_lib.geo_probe_contraction(h, int(tensor), int(zones), int(reps), _vp(out.data_ptr()), ctypes.byref(ms)),
           "geo_probe_contraction")
    return ms.value


def geo_debug_buffer(h, which, count):
    out = np.empty(count)
    _check(_lib.geo_debug_buffer(h, which, _ptr(out), count), "geo_debug_buffer")
    return out


def geo_debug_set_buffer(h, which, data):
    data = np.ascontiguousarray(data, dtype=np.float64)
    _check(_lib.geo_debug_set_buffer(h, int(which), _ptr(data), data.size), "geo_debug_set_buffer")


def geo_debug_run_stage(h, stage, dt):
    _check(_lib.geo_debug_run_stage(h, int(stage), float(dt)), "geo_debug_run_stage")


def geo_debug_stage_vjp(h, stage, dt, U, phi, g_out, n_in):
    U = np.ascontiguousarray(U, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    g_out = np.ascontiguousarray(g_out, dtype=np.float64)
    g_in = np.empty(n_in)
    _check(_lib.geo_debug_stage_vjp(h, int(stage), float(dt), _ptr(U), _ptr(phi), _ptr(g_out), g_out.size,
                                    _ptr(g_in), n_in), "geo_debug_stage_vjp")
    return g_in


def geo_cfl_dt_noalloc(h, U_dev, cfl, dt_dev):
    """Allocation-free CFL step: U_dev (8, Z) and dt_dev (1,) are caller-owned CUDA
    float64 tensors; only enqueues work on the mesh stream."""
    assert _is_device(U_dev) and _is_device(dt_dev)
    _check(_lib.geo_cfl_dt_noalloc(h, _ptr(U_dev), cfl, _ptr(dt_dev)), "geo_cfl_dt_noalloc")


def geo_step_adjoint(h, dt, U_in, phi_in, gU_out, gphi_out, gU_in, gphi_in):
    """Cotangent at t from the cotangent at t+dt (all CUDA float64 tensors)."""
    for t in (U_in, phi_in, gU_out, gphi_out, gU_in, gphi_in):
        assert _is_device(t)
    _check(_lib.geo_step_adjoint(h, dt, _ptr(U_in), _ptr(phi_in), _ptr(gU_out), _ptr(gphi_out),
                                 _ptr(gU_in), _ptr(gphi_in)), "geo_step_adjoint")


def geo_outer_Br2(h, phi_dev, gphi_dev=None):
    J = _d()
    _check(_lib.geo_outer_Br2(h, _ptr(phi_dev), ctypes.byref(J),
                              _ptr(gphi_dev) if gphi_dev is not None else None), "geo_outer_Br2")
    return J.value


def geo_last_error():
    return _lib.geo_last_error().decode()


# ---------------------------------------------------------------- convenience
class Mesh:
    """Owns one geo_mesh_t handle."""

    def __init__(self, subdiv, nr, r_in, r_out, order, prec=GEO_FP64, stream=0, gamma=5.0 / 3.0):
        self.h = geo_mesh_create(subdiv, nr, r_in, r_out, order, prec, stream)
        self.Z, self.F, self.E = geo_mesh_sizes(self.h)
        self.order = order
        self.prec = prec
        self.args = (subdiv, nr, r_in, r_out, order)
        self.stream = stream
        self.gamma = gamma
        self._adjoint_twin = None
        if gamma != 5.0 / 3.0:
            geo_set_gamma(self.h, gamma)

    def adjoint_mesh(self):
        """The mesh whose geo_step_adjoint differentiates this mesh's steps: itself
        for the FP64 form; for the FP32-bulk form an FP64 mesh of the same geometry
        (made on first use), which linearises the step about the FP32-bulk
        checkpoints."""
        if self.prec == GEO_FP64:
            return self
        if self._adjoint_twin is None:
            self._adjoint_twin = Mesh(*self.args, prec=GEO_FP64, stream=self.stream, gamma=self.gamma)
        return self._adjoint_twin

    def close(self):
        if self._adjoint_twin is not None:
            self._adjoint_twin.close()
            self._adjoint_twin = None
        if self.h:
            geo_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def initial_state(self, problem, nq_zone=None, nq_edge=8):
        """Zone averages by tensor Gauss cubature on each mapped zone and face fluxes
        from the edge circulation of the problem's vector potential."""
        nq = nq_zone or (self.order + 2)
        pts, w = geo_zone_cubature(self.h, nq)
        U = problem.zone_averages(pts, w)
        epts, tw = geo_edge_quadrature(self.h, nq_edge)
        circ = problem.edge_circulation(epts, tw)
        phi = geo_phi_from_edge_circulation(self.h, circ)
        if problem.has_radial_flux():
            n, nr = self.args[0], self.args[1]
            nrad = 6 * n * n * (nr + 1)
            fpts, wn = geo_radial_face_quadrature(self.h, nq_edge, nrad)
            phi[:nrad] += problem.radial_face_flux(fpts, wn)
        return np.ascontiguousarray(U.T), phi

    def upload(self, U, phi):
        geo_state_upload(self.h, U, phi)

    def download(self):
        U = np.empty((8, self.Z))
        phi = np.empty(self.F)
        geo_state_download(self.h, U, phi)
        return U, phi

    def step(self, dt):
        geo_step(self.h, dt)

    def cfl_dt(self, cfl):
        return geo_cfl_dt(self.h, cfl)

    def divB(self):
        return geo_divB_max(self.h)
