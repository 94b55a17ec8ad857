"""Python front end of the C ABI: tc_init / tc_layout / tc_apply / tc_energy.

Device memory and streams come from PyTorch; every computation runs in
libtc.so.  Orbital arrays are complex128 tensors of shape (Nk, nbands,
npw_max) in the layout of ``Context.layout()``.
"""
import ctypes

import numpy as np

from . import _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _data_ptr(x):
    """Pointer of a contiguous complex128 torch tensor (any device) or numpy array."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.complex128 or not x.flags.c_contiguous:
            raise TypeError("orbital arrays must be C-contiguous complex128")
        return ctypes.c_void_p(x.ctypes.data)
    if not x.is_contiguous() or str(x.dtype) != "torch.complex128":
        raise TypeError("orbital tensors must be contiguous complex128")
    return ctypes.c_void_p(x.data_ptr())


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(int(stream))


class Context:
    """One tc_init context (owns the library's tables and workspace)."""

    def __init__(self, lattice, kmesh, ecut, fft, nbands, nocc, A, C, alpha=0.0, div_correction=1,
                 ushort_factor=1.0, precision="fp64", term_mask=0):
        self.lib = _lib.load()
        self.params = _lib.make_params(lattice, kmesh, ecut, fft, nbands, nocc, A, C, alpha, div_correction,
                                       ushort_factor, precision, term_mask)
        h = ctypes.c_void_p()
        st = self.lib.tc_init(ctypes.byref(self.params), ctypes.byref(h))
        if st != _lib.TC_OK:
            msg = self.lib.tc_last_error(None)
            raise _lib.TCError(st, msg.decode() if msg else "tc_init failed")
        self.h = h
        self._finish_init(nbands, nocc)

    def _finish_init(self, nbands, nocc):
        self.nbands, self.nocc = int(nbands), int(nocc)
        nk, npw_max = ctypes.c_int(), ctypes.c_int()
        pn = ctypes.POINTER(ctypes.c_int)()
        pm = ctypes.POINTER(ctypes.c_int)()
        _lib.check(self.lib, self.h, self.lib.tc_layout(self.h, ctypes.byref(nk), ctypes.byref(npw_max),
                                                        ctypes.byref(pn), ctypes.byref(pm)))
        self.nk, self.npw_max = nk.value, npw_max.value
        self.npw = np.ctypeslib.as_array(pn, shape=(self.nk,)).copy()
        self.miller = np.ctypeslib.as_array(pm, shape=(self.nk, self.npw_max, 3)).copy()
        sc = (ctypes.c_double * 4)()
        _lib.check(self.lib, self.h, self.lib.tc_setup_scalars(self.h, sc))
        self.Omega, self.alpha, self.Gamma0, self.ndelta = sc[0], sc[1], sc[2], int(sc[3])

    def layout(self):
        return self.npw, self.miller

    def _occ(self, occ, nk=None):
        nk = self.nk if nk is None else nk
        occ = np.ascontiguousarray(np.asarray(occ, dtype=np.float64).reshape(nk, self.nbands))
        return occ, occ.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def _check_orbitals(self, x, nk=None):
        shape = (self.nk if nk is None else nk, self.nbands, self.npw_max)
        if tuple(x.shape) != shape:
            raise ValueError("orbital array must have shape %s" % (shape,))
        return x

    def apply(self, phi_R, phi_L, occ, out_R=None, out_L=None, stream=None):
        """(out_R, out_L) = operator applied to every right / left orbital (torch, cuda)."""
        import torch
        phi_R = self._check_orbitals(phi_R).contiguous()
        phi_L = self._check_orbitals(phi_L).contiguous()
        if phi_R.dtype != torch.complex128 or phi_L.dtype != torch.complex128:
            raise TypeError("orbitals must be complex128")
        if out_R is None:
            out_R = torch.empty_like(phi_R)
        if out_L is None:
            out_L = torch.empty_like(phi_L)
        occ_np, occ_p = self._occ(occ)
        st = self.lib.tc_apply(self.h, _ptr(phi_R), _ptr(phi_L), occ_p, _ptr(out_R), _ptr(out_L),
                               _stream_handle(stream))
        _lib.check(self.lib, self.h, st)
        return out_R, out_L

    def apply_host(self, phi_R, phi_L, occ, stream=None):
        """Host arrays in and out (numpy complex128): the copies run inside the call."""
        phi_R = np.ascontiguousarray(self._check_orbitals(phi_R), dtype=np.complex128)
        phi_L = np.ascontiguousarray(self._check_orbitals(phi_L), dtype=np.complex128)
        out_R = np.empty_like(phi_R)
        out_L = np.empty_like(phi_L)
        occ_np, occ_p = self._occ(occ)
        vp = ctypes.c_void_p
        st = self.lib.tc_apply(self.h, vp(phi_R.ctypes.data), vp(phi_L.ctypes.data), occ_p,
                               vp(out_R.ctypes.data), vp(out_L.ctypes.data), _stream_handle(stream))
        _lib.check(self.lib, self.h, st)
        return out_R, out_L

    def energy(self, phi_R, phi_L, occ, terms=False, stream=None):
        """TC pseudo-energy per cell; with terms=True also the per-term dict."""
        import torch
        phi_R = self._check_orbitals(phi_R).contiguous()
        phi_L = self._check_orbitals(phi_L).contiguous()
        occ_np, occ_p = self._occ(occ)
        E = ctypes.c_double()
        Et = (ctypes.c_double * _lib.TC_NTERMS)() if terms else None
        st = self.lib.tc_energy(self.h, _ptr(phi_R), _ptr(phi_L), occ_p, ctypes.byref(E),
                                Et if terms else None, _stream_handle(stream))
        _lib.check(self.lib, self.h, st)
        if not terms:
            return E.value
        d = {t: Et[i] for i, t in enumerate(_lib.TERMS)}
        d["kin"] = Et[16]
        return E.value, d

    def energy_grad(self, phi_R, phi_L, occ, orbitals=True, params=True, stream=None):
        """Gradient of energy(): (g_phi, g_chi, dE_dA[2], dE_dC[2]).

        g = dE/dRe(c) + i dE/dIm(c) for the right (phi) and left (chi) coefficients
        (torch complex128 on the orbitals' device); dE_dA, dE_dC are numpy arrays
        [parallel, antiparallel].  Skipped parts are returned as None.
        """
        import torch
        phi_R = self._check_orbitals(phi_R).contiguous()
        phi_L = self._check_orbitals(phi_L).contiguous()
        occ_np, occ_p = self._occ(occ)
        g_phi = torch.empty_like(phi_R) if orbitals else None
        g_chi = torch.empty_like(phi_L) if orbitals else None
        dA = (ctypes.c_double * 2)() if params else None
        dC = (ctypes.c_double * 2)() if params else None
        st = self.lib.tc_energy_grad(self.h, _ptr(phi_R), _ptr(phi_L), occ_p,
                                     _ptr(g_phi) if orbitals else None, _ptr(g_chi) if orbitals else None,
                                     dA, dC, _stream_handle(stream))
        _lib.check(self.lib, self.h, st)
        return (g_phi, g_chi, np.array(dA[:]) if params else None, np.array(dC[:]) if params else None)

    def biorthonormalize(self, phi_R, phi_L, stream=None):
        """In place: phi_R orthonormal (Gram-Schmidt), phi_L biorthonormal to it, per k (torch or numpy)."""
        for x in (phi_R, phi_L):
            self._check_orbitals(x)
        st = self.lib.tc_biorthonormalize(self.h, _data_ptr(phi_R), _data_ptr(phi_L), _stream_handle(stream))
        _lib.check(self.lib, self.h, st)
        return phi_R, phi_L

    def davidson_step(self, phi_R, phi_L, occ, stream=None):
        """One block-Davidson step (tc_davidson_step): (phi, chi, eig (Nk, nbands) complex, dim (Nk,)).

        Inputs and the returned orbitals are torch complex128 on the device, or numpy
        arrays (then the outputs are numpy too); eig and dim are numpy arrays.
        """
        for x in (phi_R, phi_L):
            self._check_orbitals(x)
        if isinstance(phi_R, np.ndarray):
            phi_R = np.ascontiguousarray(phi_R, dtype=np.complex128)
            phi_L = np.ascontiguousarray(phi_L, dtype=np.complex128)
            out_phi, out_chi = np.empty_like(phi_R), np.empty_like(phi_L)
        else:
            import torch
            phi_R, phi_L = phi_R.contiguous(), phi_L.contiguous()
            out_phi, out_chi = torch.empty_like(phi_R), torch.empty_like(phi_L)
        occ_np, occ_p = self._occ(occ)
        eig = np.empty((self.nk, self.nbands), dtype=np.complex128)
        dim = np.empty(self.nk, dtype=np.int32)
        st = self.lib.tc_davidson_step(self.h, _data_ptr(phi_R), _data_ptr(phi_L), occ_p, _data_ptr(out_phi),
                                       _data_ptr(out_chi), ctypes.c_void_p(eig.ctypes.data),
                                       ctypes.c_void_p(dim.ctypes.data), _stream_handle(stream))
        _lib.check(self.lib, self.h, st)
        return out_phi, out_chi, eig, dim

    def set_symmetry(self, ops, time_reversal=True):
        """Symmetry-reduced occupied-pair stage (tc_set_symmetry); ops: (nops, 3, 3) integer matrices
        acting on fractional coordinates, identity included; an empty list switches it off."""
        ops = np.ascontiguousarray(np.asarray(ops, dtype=np.int32).reshape(-1, 9))
        st = self.lib.tc_set_symmetry(self.h, ops.shape[0], ops.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      1 if time_reversal else 0)
        _lib.check(self.lib, self.h, st)

    def symmetry_info(self):
        """(number of irreducible k-points, (Nk, 6) map {k0, op, tr, K1, K2, K3})."""
        n = ctypes.c_int()
        km = np.zeros((self.nk, 6), dtype=np.int32)
        _lib.check(self.lib, self.h, self.lib.tc_symmetry_info(self.h, ctypes.byref(n),
                                                               km.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return n.value, km

    def symmetrize_orbitals(self, phi_R, phi_L, stream=None):
        """In place: orbitals of non-irreducible k-points from their irreducible points (torch or numpy)."""
        for x in (phi_R, phi_L):
            self._check_orbitals(x)
        st = self.lib.tc_symmetrize_orbitals(self.h, _data_ptr(phi_R), _data_ptr(phi_L), _stream_handle(stream))
        _lib.check(self.lib, self.h, st)
        return phi_R, phi_L

    def autotune(self, phi_R, phi_L, occ, stream=None):
        """Measure and keep the partner-chunk counts of the two-sided apply (tc_autotune): (so, sc)."""
        for x in (phi_R, phi_L):
            self._check_orbitals(x)
        occ_np, occ_p = self._occ(occ)
        so, sc = ctypes.c_int(), ctypes.c_int()
        st = self.lib.tc_autotune(self.h, _data_ptr(phi_R), _data_ptr(phi_L), occ_p, ctypes.byref(so),
                                  ctypes.byref(sc), _stream_handle(stream))
        _lib.check(self.lib, self.h, st)
        return so.value, sc.value

    def profile(self, enable=True):
        """Enable (and reset) or disable per-stage device timing."""
        _lib.check(self.lib, self.h, self.lib.tc_profile(self.h, 1 if enable else 0))

    def stage_times(self):
        """{stage: (accumulated ms, kernel launches)} since profile(True)."""
        ms = (ctypes.c_double * _lib.TC_NSTAGES)()
        nl = (ctypes.c_int * _lib.TC_NSTAGES)()
        _lib.check(self.lib, self.h, self.lib.tc_stage_times(self.h, ms, nl, _lib.TC_NSTAGES))
        return {s: (ms[i], nl[i]) for i, s in enumerate(_lib.STAGES)}

    def pair_kernels(self):
        """{stage: (kind, support, ctas)} of the pair chains, the 3b4 pass and the occupied-pair stage
        (kind 0 full transforms, 1 pruned, 2 on thread-block clusters; tc_pair_kernels)."""
        info = (ctypes.c_int * 9)()
        _lib.check(self.lib, self.h, self.lib.tc_pair_kernels(self.h, info))
        return {s: tuple(info[3 * i: 3 * i + 3]) for i, s in enumerate(("pair_chain", "pair_3b4", "occ_pairs"))}

    def pair_mirror(self):
        """(active, bytes): whether two-sided applies take the left pair spectra from the right ones
        (tc_pair_mirror)."""
        a = ctypes.c_int()
        b = ctypes.c_ulonglong()
        _lib.check(self.lib, self.h, self.lib.tc_pair_mirror(self.h, ctypes.byref(a), ctypes.byref(b)))
        return bool(a.value), int(b.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.tc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fft3d(x, sign, stream=None):
    """In-place batched 3D FFT of a (batch, n, n, n) complex cuda tensor with the library's kernel."""
    import torch
    lib = _lib.load()
    n = x.shape[-1]
    prec = _lib.TC_FP64 if x.dtype == torch.complex128 else _lib.TC_FP32
    batch = int(np.prod(x.shape[:-3])) if x.dim() > 3 else 1
    st = lib.tc_fft3d(n, prec, int(sign), _ptr(x), batch, _stream_handle(stream))
    _lib.check(lib, None, st)
    return x


def alu_peak(precision="fp32", target_ms=50.0, stream=None):
    """tc_alu_peak: measured FMA throughput (TFLOP/s) of the current device's FP32 or FP64 pipes."""
    lib = _lib.load()
    out = ctypes.c_double(0.0)
    prec = _lib.TC_FP64 if precision in ("fp64", _lib.TC_FP64) else _lib.TC_FP32
    _lib.check(lib, None, lib.tc_alu_peak(prec, float(target_ms), ctypes.byref(out), _stream_handle(stream)))
    return out.value


def band_constants(lattice, kmesh, ecut, fft, nbands, nocc, A, C, kfrac_band, alpha=0.0):
    """tc_band_constants: (gamma_b (nkb,), W (nkb, 3)) of band points kfrac_band off the SCF mesh (host only)."""
    lib = _lib.load()
    prm = _lib.make_params(lattice, kmesh, ecut, fft, nbands, nocc, A, C, alpha)
    kf = np.ascontiguousarray(np.atleast_2d(kfrac_band), dtype=np.float64)
    n = kf.shape[0]
    g = np.zeros(n)
    W = np.zeros((n, 3))
    dp = ctypes.POINTER(ctypes.c_double)
    st = lib.tc_band_constants(ctypes.byref(prm), kf.ctypes.data_as(dp), n, g.ctypes.data_as(dp),
                               W.ctypes.data_as(dp))
    _lib.check(lib, None, st)
    return g, W


def band_layout(lattice, kmesh, ecut, fft, nbands, nocc, A, C, kfrac_band):
    """tc_band_layout: (npw (nkb,), miller (nkb, max npw, 3)) of the spheres at band points kfrac_band."""
    lib = _lib.load()
    prm = _lib.make_params(lattice, kmesh, ecut, fft, nbands, nocc, A, C)
    kf = np.ascontiguousarray(np.atleast_2d(kfrac_band), dtype=np.float64)
    n = kf.shape[0]
    npw = np.zeros(n, dtype=np.int32)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    _lib.check(lib, None, lib.tc_band_layout(ctypes.byref(prm), kf.ctypes.data_as(dp), n, 0, npw.ctypes.data_as(ip),
                                             None))
    m = max(int(npw.max()) if n else 0, 1)
    miller = np.zeros((n, m, 3), dtype=np.int32)
    _lib.check(lib, None, lib.tc_band_layout(ctypes.byref(prm), kf.ctypes.data_as(dp), n, m, npw.ctypes.data_as(ip),
                                             miller.ctypes.data_as(ip)))
    return npw, miller


class BandContext(Context):
    """tc_init_band: the operator at band points kfrac_band off the SCF mesh (partners on the mesh).

    ``layout()`` covers the Nk mesh points then the nkb band points with one npw_max; mesh and
    band-point orbital arrays both use it.
    """

    def __init__(self, lattice, kmesh, ecut, fft, nbands, nocc, A, C, kfrac_band, alpha=0.0, div_correction=1,
                 ushort_factor=1.0, precision="fp64", term_mask=0):
        self.lib = _lib.load()
        self.params = _lib.make_params(lattice, kmesh, ecut, fft, nbands, nocc, A, C, alpha, div_correction,
                                       ushort_factor, precision, term_mask)
        kf = np.ascontiguousarray(np.atleast_2d(kfrac_band), dtype=np.float64)
        self.nkb = kf.shape[0]
        h = ctypes.c_void_p()
        st = self.lib.tc_init_band(ctypes.byref(self.params), self.nkb, kf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.byref(h))
        if st != _lib.TC_OK:
            msg = self.lib.tc_last_error(None)
            raise _lib.TCError(st, msg.decode() if msg else "tc_init_band failed")
        self.h = h
        self._finish_init(nbands, nocc)
        self.nk_mesh = self.nk - self.nkb

    def apply_band(self, phi_R, phi_L, occ, band_phi_R, band_phi_L, band_occ, out_R=None, out_L=None, stream=None):
        """(out_R, out_L) at the band points, [nkb][nbands][npw_max] complex128 on the orbitals' device."""
        import torch
        arrs = [self._check_orbitals(x, self.nk_mesh).contiguous() for x in (phi_R, phi_L)]
        barrs = [self._check_orbitals(x, self.nkb).contiguous() for x in (band_phi_R, band_phi_L)]
        occ_np, occ_p = self._occ(occ, self.nk_mesh)
        bocc_np, bocc_p = self._occ(band_occ, self.nkb)
        if out_R is None:
            out_R = torch.empty_like(barrs[0])
        if out_L is None:
            out_L = torch.empty_like(barrs[1])
        st = self.lib.tc_apply_band(self.h, _ptr(arrs[0]), _ptr(arrs[1]), occ_p, _ptr(barrs[0]), _ptr(barrs[1]), bocc_p,
                                    _ptr(out_R), _ptr(out_L), _stream_handle(stream))
        _lib.check(self.lib, self.h, st)
        return out_R, out_L


class BatchContext:
    """tc_init_batch: many independent cells sharing one workspace, applied by one graph launch.

    ``cells`` is a list of dicts with the Context arguments (lattice, kmesh, ecut,
    fft, nbands, nocc, A, C and optionally alpha, div_correction, ushort_factor,
    term_mask); every cell uses ``precision``.
    """

    def __init__(self, cells, precision="fp32"):
        self.lib = _lib.load()
        keys = ("lattice", "kmesh", "ecut", "fft", "nbands", "nocc", "A", "C")
        opt = ("alpha", "div_correction", "ushort_factor", "term_mask")
        prm = [_lib.make_params(*[c[k] for k in keys], **{k: c[k] for k in opt if k in c}, precision=precision)
               for c in cells]
        self.params = (_lib.tc_params * len(prm))(*prm)
        h = ctypes.c_void_p()
        st = self.lib.tc_init_batch(len(prm), self.params, ctypes.byref(h))
        if st != _lib.TC_OK:
            msg = self.lib.tc_last_error(None)
            raise _lib.TCError(st, msg.decode() if msg else "tc_init_batch failed")
        self.h = h
        self.ncell = len(prm)
        self.layouts = []
        for i in range(self.ncell):
            ch = ctypes.c_void_p()
            _lib.check(self.lib, self.h, self.lib.tc_batch_cell(self.h, i, ctypes.byref(ch)))
            nk, npw_max = ctypes.c_int(), ctypes.c_int()
            pn = ctypes.POINTER(ctypes.c_int)()
            pm = ctypes.POINTER(ctypes.c_int)()
            _lib.check(self.lib, ch, self.lib.tc_layout(ch, ctypes.byref(nk), ctypes.byref(npw_max), ctypes.byref(pn),
                                                        ctypes.byref(pm)))
            npw = np.ctypeslib.as_array(pn, shape=(nk.value,)).copy()
            miller = np.ctypeslib.as_array(pm, shape=(nk.value, npw_max.value, 3)).copy()
            self.layouts.append((nk.value, npw_max.value, npw, miller))

    def apply(self, phi_R, phi_L, occ, out_R=None, out_L=None, stream=None):
        """Lists of per-cell complex128 cuda tensors in, lists out (both operator sides)."""
        import torch
        n = self.ncell
        out_R = out_R if out_R is not None else [torch.empty_like(x) for x in phi_R]
        out_L = out_L if out_L is not None else [torch.empty_like(x) for x in phi_L]
        vp = ctypes.c_void_p
        occs = [np.ascontiguousarray(np.asarray(o, dtype=np.float64)) for o in occ]
        dpp = ctypes.POINTER(ctypes.c_double)
        arrs = [(vp * n)(*[vp(x.data_ptr()) for x in xs]) for xs in (phi_R, phi_L, out_R, out_L)]
        occ_arr = (dpp * n)(*[o.ctypes.data_as(dpp) for o in occs])
        st = self.lib.tc_apply_batch(self.h, arrs[0], arrs[1], occ_arr, arrs[2], arrs[3], _stream_handle(stream))
        _lib.check(self.lib, self.h, st)
        return out_R, out_L

    def info(self):
        """(ncell, chosen lanes, largest lane count, {lanes: measured replay ms})."""
        nc, ln, lm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_double * 5)()
        _lib.check(self.lib, self.h, self.lib.tc_batch_info(self.h, ctypes.byref(nc), ctypes.byref(ln),
                                                            ctypes.byref(lm), ms))
        return nc.value, ln.value, lm.value, {L: ms[i] for i, L in enumerate((1, 2, 4, 8, 16)) if ms[i] >= 0}

    def close(self):
        if getattr(self, "h", None):
            self.lib.tc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
