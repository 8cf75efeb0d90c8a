"""ctypes declarations of the C ABI in include/lf.h (argument marshalling only).

The shared library is built in-tree (paper_2609_08649_b300/liblf.so).  There is no
fallback: if the library is missing or fails to load, importing the binding raises.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LF_LIBRARY") or os.path.join(HERE, "liblf.so")

LF_OK, LF_EINVAL, LF_ECUDA, LF_ENOMEM, LF_ETIMEOUT, LF_EUNSUPPORTED = range(6)
LF_SIE, LF_DPIE, LF_NFW, LF_SHEAR = 1, 2, 3, 4
LF_FP64, LF_MIXED, LF_FF = 0, 1, 2
STATUS_NAMES = {0: "LF_OK", 1: "LF_EINVAL", 2: "LF_ECUDA", 3: "LF_ENOMEM", 4: "LF_ETIMEOUT",
                5: "LF_EUNSUPPORTED"}


class lf_comp(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("b", C.c_double), ("eps", C.c_double),
                ("pa", C.c_double), ("core", C.c_double), ("cut", C.c_double),
                ("kind", C.c_int32), ("pad", C.c_int32)]


class lf_member(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("log_l", C.c_double), ("pad", C.c_double)]


class lf_scaling(C.Structure):
    _fields_ = [("b_star", C.c_double), ("core_star", C.c_double), ("cut_star", C.c_double),
                ("lam", C.c_double), ("beta", C.c_double), ("alpha", C.c_double)]


class lf_plane(C.Structure):
    _fields_ = [("n_comp", C.c_int32), ("n_mem", C.c_int32), ("comp", C.c_void_p),
                ("mem", C.c_void_p), ("scaling", lf_scaling)]


class lf_phys_comp(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("x", C.c_double), ("y", C.c_double),
                ("vdisp", C.c_double), ("theta_e", C.c_double), ("z_ref", C.c_double),
                ("eps", C.c_double), ("pa_deg", C.c_double), ("core_kpc", C.c_double),
                ("core_arcsec", C.c_double), ("cut_kpc", C.c_double), ("m200", C.c_double),
                ("conc", C.c_double), ("kappa_s", C.c_double), ("theta_s", C.c_double),
                ("gamma", C.c_double), ("amp", C.c_double)]


class lf_grid(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32)]


class lf_images(C.Structure):
    _fields_ = [("n_img", C.c_int32), ("n_fam", C.c_int32), ("theta_obs", C.c_void_p),
                ("sinv", C.c_void_p), ("fam_off", C.c_void_p), ("fam_ratio", C.c_void_p),
                ("mag", C.c_void_p), ("mag_err", C.c_void_p), ("td", C.c_void_p),
                ("td_err", C.c_void_p), ("td_scale", C.c_double)]


class lf_cluster(C.Structure):
    _fields_ = [("n_planes", C.c_int32), ("planes", C.c_void_p), ("ratios", C.c_void_p),
                ("arcsec_per_kpc", C.c_void_p), ("images", lf_images), ("P", C.c_int32),
                ("p_comp", C.c_void_p), ("p_field", C.c_void_p), ("p_xform", C.c_void_p)]


assert C.sizeof(lf_comp) == 64 and C.sizeof(lf_member) == 32


class LFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2609_08649_b300/build.py)")
    lib = C.CDLL(LIB_PATH)
    vp, i32, f64 = C.c_void_p, C.c_int32, C.c_double
    sig = {
        "lf_deflect_grid": [vp, vp, i32, vp, vp, vp],
        "lf_jacobian_grid": [vp, vp, f64, i32, vp, vp, vp, vp, vp, vp, vp],
        "lf_jacobian_points": [vp, vp, i32, f64, i32, vp, vp, vp, vp, vp, vp, vp],
        "lf_jacobian_grid_host": [vp, vp, f64, i32, vp, vp, vp, vp, vp, vp, i32, vp, C.c_size_t, vp],
        "lf_trace_multiplane": [vp, i32, vp, vp, i32, vp, i32, vp, vp, vp],
        "lf_plan_create": [vp, vp, i32, i32, i32, i32],
        "lf_chi2_batch": [vp, vp, i32, vp, vp],
        "lf_chi2_grad_batch": [vp, vp, i32, vp, vp, vp],
        "lf_plan_destroy": [vp],
        "lf_chi2_img_batch": [vp, vp, i32, i32, vp, vp, vp],
        "lf_aies_run": [vp, vp, vp, i32, i32, vp, f64, vp, vp, vp, vp, vp],
        "lf_mh_run": [vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp],
        "lf_nm_run": [vp, vp, vp, i32, i32, vp, vp, vp, vp],
        "lf_probe_alu": [vp, vp, vp, vp],
        "lf_probe_alu2": [vp, vp, vp, vp, vp],
        "lf_selftest_wait_timeout": [C.c_uint32, vp],
        "lf_chi2_batch_static": [vp, vp, i32, i32, vp, vp],
        "lf_plan_info": [vp, vp, vp, vp],
        "lf_nfw_params": [f64, f64, f64, f64, f64, vp, vp],
        "lf_comp_from_physical": [vp, f64, f64, f64, vp],
        "lf_scaling_from_physical": [f64] * 9 + [vp],
        "lf_multiplane_ratios": [f64, f64, vp, i32, f64, vp],
        "lf_device_error": [vp],
        "lf_find_images": [vp, vp, i32, vp, vp, i32, i32, i32, vp, C.c_size_t, vp, vp, vp],
        "lf_find_images_multiplane": [vp, i32, vp, vp, i32, vp, i32, i32, i32, vp, C.c_size_t, vp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    for name, args in {"lf_angular_distance": [f64] * 4, "lf_adis": [f64] * 4,
                       "lf_arcsec_per_kpc": [f64] * 3, "lf_b_from_vdisp": [f64],
                       "lf_td_scale": [f64] * 3}.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_double
    lib.lf_jacobian_grid_host_workspace.argtypes = [vp, i32]
    lib.lf_jacobian_grid_host_workspace.restype = C.c_size_t
    lib.lf_find_images_workspace.argtypes = [i32, i32, i32, i32]
    lib.lf_find_images_workspace.restype = C.c_size_t
    lib.lf_find_images_multiplane_workspace.argtypes = [i32, i32, i32, i32]
    lib.lf_find_images_multiplane_workspace.restype = C.c_size_t
    lib.lf_last_error.restype = C.c_char_p
    lib.lf_version.restype = C.c_char_p
    return lib


lib = _load()

# Every symbol the header declares (checked by the CPU test-suite).
EXPORTS = ["lf_deflect_grid", "lf_jacobian_grid", "lf_jacobian_grid_host", "lf_jacobian_grid_host_workspace",
           "lf_jacobian_points", "lf_trace_multiplane",
           "lf_plan_create", "lf_chi2_batch", "lf_chi2_grad_batch", "lf_plan_destroy",
           "lf_chi2_img_batch", "lf_aies_run", "lf_mh_run", "lf_nm_run", "lf_find_images", "lf_find_images_workspace", "lf_find_images_multiplane",
           "lf_find_images_multiplane_workspace",
           "lf_chi2_batch_static",
           "lf_plan_info", "lf_angular_distance", "lf_adis", "lf_arcsec_per_kpc",
           "lf_b_from_vdisp", "lf_td_scale", "lf_nfw_params", "lf_comp_from_physical", "lf_scaling_from_physical",
           "lf_multiplane_ratios", "lf_device_error", "lf_selftest_wait_timeout", "lf_probe_alu", "lf_probe_alu2", "lf_last_error", "lf_version"]


def check(status):
    if status != LF_OK:
        raise LFError(status, lib.lf_last_error().decode())
    return status
