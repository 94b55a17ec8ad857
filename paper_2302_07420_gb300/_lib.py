"""ctypes binding of libtc.so (include/tc.h): argument marshalling only.

Every step of the operator runs in the CUDA library; this module converts
arguments and raises on a non-OK status.  It fails loudly if the in-tree
library is missing -- there is no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtc.so")

(TC_OK, TC_ERR_ARG, TC_ERR_STATE, TC_ERR_OOM, TC_ERR_CUDA, TC_ERR_TIMEOUT, TC_ERR_UNSUPPORTED,
 TC_ERR_NUMERIC) = range(8)
TC_FP64, TC_FP32, TC_FP32_COMP, TC_BF16_STORE = 0, 1, 2, 3
PRECISIONS = {"fp64": TC_FP64, "fp32": TC_FP32, "fp32_comp": TC_FP32_COMP, "bf16_store": TC_BF16_STORE}
TERMS = ("2ah", "2bh1", "2bh2", "2ax", "2bx1", "2bx2", "3a1", "3a2", "3a3", "3a4",
         "3b1", "3b2", "3b3", "3b4", "3b5", "3b6")
TC_NTERMS = 17          # 16 operator terms + kinetic
EXPORTED = ("tc_init", "tc_layout", "tc_setup_scalars", "tc_apply", "tc_energy", "tc_fft3d",
            "tc_last_error", "tc_destroy", "tc_profile", "tc_stage_times", "tc_apply_noalloc", "tc_energy_grad",
            "tc_biorthonormalize", "tc_init_batch", "tc_batch_cell", "tc_apply_batch", "tc_batch_info",
            "tc_davidson_step", "tc_set_symmetry", "tc_symmetry_info", "tc_symmetrize_orbitals", "tc_autotune",
            "tc_alu_peak", "tc_band_constants", "tc_band_layout", "tc_init_band", "tc_apply_band",
            "tc_pair_kernels", "tc_pair_mirror")
TC_NSTAGES = 6
STAGES = ("orbitals", "hartree", "occ_pairs", "pair_chain", "pair_3b4", "finalize")
STATUS = {TC_ERR_ARG: "TC_ERR_ARG", TC_ERR_STATE: "TC_ERR_STATE", TC_ERR_OOM: "TC_ERR_OOM",
          TC_ERR_CUDA: "TC_ERR_CUDA", TC_ERR_TIMEOUT: "TC_ERR_TIMEOUT", TC_ERR_UNSUPPORTED: "TC_ERR_UNSUPPORTED",
          TC_ERR_NUMERIC: "TC_ERR_NUMERIC"}


class tc_params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_double * 9),
        ("kmesh", ctypes.c_int * 3),
        ("ecut_ha", ctypes.c_double),
        ("fft", ctypes.c_int * 3),
        ("nbands", ctypes.c_int),
        ("nocc", ctypes.c_int),
        ("A", ctypes.c_double * 2),
        ("C", ctypes.c_double * 2),
        ("alpha", ctypes.c_double),
        ("div_correction", ctypes.c_int),
        ("ushort_factor", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("term_mask", ctypes.c_uint),
    ]


class TCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None


def load():
    """Load the in-tree CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libtc.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2302_07420_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip = ctypes.c_void_p, ctypes.c_int
    lib.tc_init.argtypes = [ctypes.POINTER(tc_params), ctypes.POINTER(vp)]
    lib.tc_layout.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ctypes.POINTER(ip)),
                              ctypes.POINTER(ctypes.POINTER(ip))]
    lib.tc_setup_scalars.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.tc_apply.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp, vp, vp]
    lib.tc_energy.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double), vp]
    lib.tc_fft3d.argtypes = [ip, ip, ip, vp, ip, vp]
    lib.tc_last_error.argtypes = [vp]
    lib.tc_last_error.restype = ctypes.c_char_p
    lib.tc_destroy.argtypes = [vp]
    lib.tc_profile.argtypes = [vp, ip]
    lib.tc_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ip), ip]
    lib.tc_apply_noalloc.argtypes = [ctypes.POINTER(tc_params), vp, vp, ctypes.POINTER(ctypes.c_double), vp, vp, vp]
    dp = ctypes.POINTER(ctypes.c_double)
    lib.tc_energy_grad.argtypes = [vp, vp, vp, dp, vp, vp, dp, dp, vp]
    lib.tc_biorthonormalize.argtypes = [vp, vp, vp, vp]
    lib.tc_init_batch.argtypes = [ip, ctypes.POINTER(tc_params), ctypes.POINTER(vp)]
    lib.tc_batch_cell.argtypes = [vp, ip, ctypes.POINTER(vp)]
    lib.tc_apply_batch.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(dp),
                                   ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.tc_batch_info.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip), dp]
    lib.tc_davidson_step.argtypes = [vp, vp, vp, dp, vp, vp, vp, vp, vp]
    lib.tc_set_symmetry.argtypes = [vp, ip, ctypes.POINTER(ip), ip]
    lib.tc_symmetry_info.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip)]
    lib.tc_symmetrize_orbitals.argtypes = [vp, vp, vp, vp]
    lib.tc_autotune.argtypes = [vp, vp, vp, dp, ctypes.POINTER(ip), ctypes.POINTER(ip), vp]
    lib.tc_alu_peak.argtypes = [ip, ctypes.c_double, dp, vp]
    lib.tc_band_constants.argtypes = [ctypes.POINTER(tc_params), dp, ip, dp, dp]
    lib.tc_band_layout.argtypes = [ctypes.POINTER(tc_params), dp, ip, ip, ctypes.POINTER(ip), ctypes.POINTER(ip)]
    lib.tc_init_band.argtypes = [ctypes.POINTER(tc_params), ip, dp, ctypes.POINTER(vp)]
    lib.tc_apply_band.argtypes = [vp, vp, vp, dp, vp, vp, dp, vp, vp, vp]
    lib.tc_pair_mirror.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ctypes.c_ulonglong)]
    for name in ("tc_init_band", "tc_apply_band", "tc_init", "tc_layout", "tc_setup_scalars", "tc_apply", "tc_energy", "tc_fft3d", "tc_destroy",
                 "tc_profile", "tc_stage_times", "tc_apply_noalloc", "tc_energy_grad",
            "tc_biorthonormalize", "tc_init_batch", "tc_batch_cell", "tc_apply_batch", "tc_batch_info",
            "tc_davidson_step", "tc_set_symmetry", "tc_symmetry_info", "tc_symmetrize_orbitals", "tc_autotune",
            "tc_alu_peak", "tc_band_constants", "tc_band_layout", "tc_pair_mirror"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def make_params(lattice, kmesh, ecut, fft, nbands, nocc, A, C, alpha=0.0, div_correction=1,
                ushort_factor=1.0, precision="fp64", term_mask=0):
    p = tc_params()
    flat = [float(x) for row in lattice for x in row]
    p.lattice = (ctypes.c_double * 9)(*flat)
    p.kmesh = (ctypes.c_int * 3)(*[int(x) for x in kmesh])
    p.ecut_ha = float(ecut)
    p.fft = (ctypes.c_int * 3)(*[int(x) for x in fft])
    p.nbands, p.nocc = int(nbands), int(nocc)
    p.A = (ctypes.c_double * 2)(*[float(x) for x in A])
    p.C = (ctypes.c_double * 2)(*[float(x) for x in C])
    p.alpha = float(alpha)
    p.div_correction = int(div_correction)
    p.ushort_factor = float(ushort_factor)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.term_mask = int(term_mask)
    return p


def check(lib, ctx, status):
    if status != TC_OK:
        msg = lib.tc_last_error(ctx)
        raise TCError(status, msg.decode() if msg else "")
