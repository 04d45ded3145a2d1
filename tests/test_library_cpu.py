"""Host-side checks of libpsf (no GPU needed): the library builds for sm_103a,
loads, exports every function include/psf.h declares, and rejects bad
arguments on the host before touching the device."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

from paper_2502_03170_gb300 import _lib, api
from paper_2502_03170_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(psf_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def cpu_lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2502_03170_gb300 import build
    build.build()
    return _lib.load()


def test_exports_every_declared_symbol(cpu_lib):
    names = declared_functions()
    assert "psf_fourier_vectorial" in names and "psf_bessel_vectorial" in names
    for n in sorted(names):
        assert hasattr(cpu_lib, n), n
    assert set(_lib.PROTOTYPES) == names
    assert cpu_lib.psf_version() >= 100


def test_host_validation(cpu_lib):
    o = api.make_optics(W.optics_plain())
    g = api.Grid(dict(nx=8, ny=8, dx=0.02, dy=0.02, z=[0.0, 0.1]))
    size = cpu_lib.psf_fourier_workspace_size(ctypes.byref(o), 16,
                                              ctypes.byref(g.c), 0)
    assert size > 0
    bad = api.make_optics(dict(W.optics_plain(), NA=1.6))
    assert cpu_lib.psf_fourier_workspace_size(ctypes.byref(bad), 16,
                                              ctypes.byref(g.c), 0) == 0
    # NA >= n_i is rejected before any launch
    r = cpu_lib.psf_fourier_vectorial(ctypes.byref(bad), 16, ctypes.byref(g.c),
                                      None, 0, None, 0, ctypes.c_void_p(16),
                                      None, ctypes.c_void_p(256), 1 << 30, None)
    assert r == _lib.PSF_ERR_ARG
    assert b"NA" in cpu_lib.psf_last_error()
    # missing intensity, too-small workspace, unknown precision
    assert cpu_lib.psf_fourier_vectorial(ctypes.byref(o), 16, ctypes.byref(g.c),
                                         None, 0, None, 0, None, None,
                                         ctypes.c_void_p(256), 1 << 30,
                                         None) == _lib.PSF_ERR_ARG
    assert cpu_lib.psf_fourier_vectorial(ctypes.byref(o), 16, ctypes.byref(g.c),
                                         None, 0, None, 0, ctypes.c_void_p(16),
                                         None, ctypes.c_void_p(256), 64,
                                         None) == _lib.PSF_ERR_WORKSPACE
    assert cpu_lib.psf_fourier_vectorial(ctypes.byref(o), 16, ctypes.byref(g.c),
                                         None, 0, None, 7, ctypes.c_void_p(16),
                                         None, ctypes.c_void_p(256), 1 << 30,
                                         None) == _lib.PSF_ERR_PRECISION
    zbad = np.zeros(67)
    assert cpu_lib.psf_fourier_vectorial(
        ctypes.byref(o), 16, ctypes.byref(g.c), zbad.ctypes.data_as(ctypes.c_void_p),
        67, None, 0, ctypes.c_void_p(16), None, ctypes.c_void_p(256), 1 << 30,
        None) == _lib.PSF_ERR_ARG
    # Bessel: n_theta out of range, non-FP32 precision
    assert cpu_lib.psf_bessel_workspace_size(ctypes.byref(o), 4, 16, 1, 64, 8,
                                             8, 0) == 0
    assert cpu_lib.psf_bessel_workspace_size(ctypes.byref(o), 4, 16, 64, 64,
                                             8, 8, 0) > 0
    r = cpu_lib.psf_bessel_vectorial(ctypes.byref(o), 4, None, None, 0, None, None,
                                     None, 16, 64, 64, 8, 8, 0.02, 0.02, 0,
                                     ctypes.c_void_p(16), None,
                                     ctypes.c_void_p(256), 1 << 30, None)
    assert r == _lib.PSF_ERR_ARG
    # Bessel backward: precision modes, grid limit, needs a target or dL/dI
    assert cpu_lib.psf_bessel_backward_workspace_size(ctypes.byref(o), 4, 16, 64,
                                                      64, 8, 8, 0) > 0
    assert cpu_lib.psf_bessel_backward_workspace_size(ctypes.byref(o), 4, 16, 64,
                                                      64, 8, 8, 1) > 0
    assert cpu_lib.psf_bessel_backward_workspace_size(ctypes.byref(o), 4, 16, 64,
                                                      64, 8, 8, 7) == 0
    assert cpu_lib.psf_bessel_backward_workspace_size(ctypes.byref(o), 4, 16, 64,
                                                      64, 8192, 8, 0) == 0
    d = ctypes.c_void_p(16)
    args = [ctypes.byref(o), 4, d, None, 0, None, d, d, 16, 64, 64, 8, 8, 0.02,
            0.02]
    tail = [ctypes.c_void_p(256), 1 << 30, None]
    assert cpu_lib.psf_bessel_vectorial_backward(
        *args, 7, d, None, None, None, None, None, *tail) == _lib.PSF_ERR_PRECISION
    assert cpu_lib.psf_bessel_vectorial_backward(
        *args, 0, None, None, None, None, None, None, *tail) == _lib.PSF_ERR_ARG
    assert cpu_lib.psf_bessel_vectorial_backward(
        *args, 0, None, d, d, None, None, None, *tail) == _lib.PSF_ERR_ARG   # loss w/o target
    # backward: needs a target or an upstream gradient
    r = cpu_lib.psf_fourier_vectorial_backward(
        ctypes.byref(o), 16, ctypes.byref(g.c), 1, None, 0, None, 0, None,
        None, None, ctypes.c_void_p(16), None, ctypes.c_void_p(256), 1 << 30,
        None)
    assert r == _lib.PSF_ERR_ARG


def test_chirpz_mode_validation(cpu_lib):
    """The chirp-Z mode: forward only, FFT length per direction <= 4096."""
    o = api.make_optics(W.optics_plain())
    C = _lib.PSF_PREC_FP32_CHIRPZ
    g = api.Grid(dict(nx=512, ny=512, dx=0.01, dy=0.01, z=[0.0, 0.1]))
    size = cpu_lib.psf_fourier_workspace_size(ctypes.byref(o), 256, ctypes.byref(g.c), C)
    # tables (2 x (2 L + N + n) + N/2 words) and the stage-1 chunk, two planes
    assert size >= 2 * 3 * 512 * 256 * 8
    assert cpu_lib.psf_fourier_backward_workspace_size(ctypes.byref(o), 256,
                                                       ctypes.byref(g.c), C) == 0
    r = cpu_lib.psf_fourier_vectorial_backward(
        ctypes.byref(o), 256, ctypes.byref(g.c), 1, None, 0, None, C,
        ctypes.c_void_p(16), None, None, ctypes.c_void_p(16), None,
        ctypes.c_void_p(256), 1 << 30, None)
    assert r == _lib.PSF_ERR_PRECISION
    assert b"forward only" in cpu_lib.psf_last_error()
    # N + n - 1 = 4096 fits, 4097 does not
    ok = api.Grid(dict(nx=2049, ny=8, dx=0.01, dy=0.01, z=[0.0]))
    assert cpu_lib.psf_fourier_workspace_size(ctypes.byref(o), 2048, ctypes.byref(ok.c), C) > 0
    big = api.Grid(dict(nx=2050, ny=8, dx=0.01, dy=0.01, z=[0.0]))
    assert cpu_lib.psf_fourier_workspace_size(ctypes.byref(o), 2048, ctypes.byref(big.c), C) == 0
    r = cpu_lib.psf_fourier_vectorial(ctypes.byref(o), 2048, ctypes.byref(big.c), None, 0,
                                      None, C, ctypes.c_void_p(16), None,
                                      ctypes.c_void_p(256), 1 << 40, None)
    assert r == _lib.PSF_ERR_PRECISION
    assert b"chirp-Z" in cpu_lib.psf_last_error()


def test_harmonic_order_and_validation(cpu_lib):
    """The truncation order of the library's host helper is the tail bound
    the oracle states; argument checks run before any launch."""
    from oracle import bessel_harmonic as bh
    c = W.bessel(n_emitters=40)
    zs = np.ascontiguousarray(c["zernike"], dtype=np.float64)
    for tol in (1e-5, 1e-7, 1e-9):
        m = cpu_lib.psf_bessel_harmonic_order(zs.ctypes.data_as(ctypes.c_void_p),
                                              zs.shape[0], zs.shape[1], tol)
        assert m == max(bh.harmonic_order(z, tol) for z in zs)
    assert cpu_lib.psf_bessel_harmonic_order(None, 0, 0, 1e-7) == 0
    assert cpu_lib.psf_bessel_harmonic_order(zs.ctypes.data_as(ctypes.c_void_p), 4,
                                             zs.shape[1], 0.0) == _lib.PSF_ERR_ARG
    o = api.make_optics(W.optics_plain())
    for prec in (_lib.PSF_PREC_FP32, _lib.PSF_PREC_SPLIT_FP16):
        assert cpu_lib.psf_bessel_harmonic_workspace_size(ctypes.byref(o), 4, 16, 64, 64,
                                                          8, 8, 12, prec) > 0
    assert cpu_lib.psf_bessel_harmonic_workspace_size(ctypes.byref(o), 4, 16, 64, 64, 8, 8,
                                                      12, _lib.PSF_PREC_SPLIT_BF16) == 0
    assert cpu_lib.psf_bessel_harmonic_workspace_size(ctypes.byref(o), 4, 16, 64, 64,
                                                      8, 8, 65, _lib.PSF_PREC_FP32) == 0
    assert cpu_lib.psf_bessel_harmonic_workspace_size(ctypes.byref(o), 4, 16, 64, 64, 8, 8,
                                                      12, _lib.PSF_PREC_FP32_CHIRPZ) == 0
    d = ctypes.c_void_p(16)
    r = cpu_lib.psf_bessel_vectorial_harmonic(ctypes.byref(o), 4, d, d, 21, d, d, 16, 64,
                                              64, 8, 8, 0.02, 0.02, -1, 0.0,
                                              _lib.PSF_PREC_FP32, d, ctypes.c_void_p(256),
                                              1 << 30, None)
    assert r == _lib.PSF_ERR_ARG
    r = cpu_lib.psf_bessel_vectorial_harmonic(ctypes.byref(o), 4, d, d, 21, d, d, 16, 64,
                                              64, 8, 8, 0.02, 0.02, 12, 0.0,
                                              _lib.PSF_PREC_FP32_CHIRPZ, d,
                                              ctypes.c_void_p(256), 1 << 30, None)
    assert r == _lib.PSF_ERR_PRECISION
    for bad in (-1e-9, 1.0, float("nan")):
        r = cpu_lib.psf_bessel_vectorial_harmonic(ctypes.byref(o), 4, d, d, 21, d, d, 16, 64,
                                                  64, 8, 8, 0.02, 0.02, 12, bad,
                                                  _lib.PSF_PREC_FP32, d, ctypes.c_void_p(256),
                                                  1 << 30, None)
        assert r == _lib.PSF_ERR_ARG and b"tail_tol" in cpu_lib.psf_last_error(), bad


def test_backward_batch_workspace(cpu_lib):
    """The batch-sized adjoint workspace grows with the batch up to its cap
    and never falls below the default one."""
    o = api.make_optics(W.optics_plain())
    g = api.Grid(dict(nx=128, ny=128, dx=0.02, dy=0.02, z=np.linspace(-1, 1, 32)))
    base = cpu_lib.psf_fourier_backward_workspace_size(ctypes.byref(o), 256, ctypes.byref(g.c), 1)
    sizes = [cpu_lib.psf_fourier_backward_workspace_size_batch(ctypes.byref(o), 256,
                                                               ctypes.byref(g.c), 1, b)
             for b in (1, 4, 16, 64, 128)]
    assert base > 0 and all(x > 0 for x in sizes)
    assert sizes[0] <= base and sizes[1] == base          # 4 x 32 = 128 planes
    assert sizes[1] < sizes[2] < sizes[3] == sizes[4]     # capped at 2048 planes
    assert cpu_lib.psf_fourier_backward_workspace_size_batch(ctypes.byref(o), 256,
                                                             ctypes.byref(g.c), 1, 0) == 0


def test_split_precision_envelope(cpu_lib):
    """Forward calls in a split mode are refused (PSF_ERR_PRECISION, before
    any launch) outside the sizes where the split contractions stay within
    the 1e-5 bound; PSF_PREC_AUTO then takes a mode that does, and the
    adjoints (gradient bound 1e-4) keep every mode."""
    o = api.make_optics(W.optics_gibson_lanni(2.0))
    g = api.Grid(dict(nx=64, ny=64, dx=0.01, dy=0.01, z=[0.0, 0.5]))
    size = lambda N, p: cpu_lib.psf_fourier_workspace_size(ctypes.byref(o), N,
                                                           ctypes.byref(g.c), p)
    F16, B16 = _lib.PSF_PREC_SPLIT_FP16, _lib.PSF_PREC_SPLIT_BF16
    assert size(512, F16) > 0 and size(1024, B16) > 0
    assert size(1024, F16) == 0
    assert b"split FP16" in cpu_lib.psf_last_error() and b"512" in cpu_lib.psf_last_error()
    assert size(2048, B16) == 0 and b"split BF16" in cpu_lib.psf_last_error()
    # AUTO: the split form's own size where it is inside, another mode beyond
    for N, mode in ((256, F16), (1024, B16), (1536, _lib.PSF_PREC_FP32_CHIRPZ),
                    (4096, _lib.PSF_PREC_FP32)):
        assert size(N, _lib.PSF_PREC_AUTO) == size(N, mode), N
    # 3xTF32 up to 256; single-pass TF32 only with PSF_OUTSIDE_ENVELOPE
    T3, T1 = _lib.PSF_PREC_SPLIT_TF32, _lib.PSF_PREC_TF32
    assert size(256, T3) > 0 and size(512, T3) == 0
    assert size(256, T1) == 0 and b"TF32" in cpu_lib.psf_last_error()
    oo = api.make_optics(dict(W.optics_gibson_lanni(2.0), outside_envelope=True))
    assert cpu_lib.psf_fourier_workspace_size(ctypes.byref(oo), 256, ctypes.byref(g.c), T1) > 0
    assert cpu_lib.psf_fourier_workspace_size(ctypes.byref(oo), 1024, ctypes.byref(g.c),
                                              F16) > 0
    # TF32 operands are 4-byte parts: twice the split FP16 operand bytes
    assert size(256, T3) > size(256, F16)
    assert cpu_lib.psf_fourier_backward_workspace_size(ctypes.byref(o), 256,
                                                       ctypes.byref(g.c), T3) == 0
    r = cpu_lib.psf_fourier_vectorial(ctypes.byref(o), 1024, ctypes.byref(g.c), None, 0,
                                      None, F16, ctypes.c_void_p(16), None,
                                      ctypes.c_void_p(256), 1 << 40, None)
    assert r == _lib.PSF_ERR_PRECISION
    # the adjoint takes split FP16 at any pupil its tensor-core form runs
    assert cpu_lib.psf_fourier_backward_workspace_size(ctypes.byref(o), 1024,
                                                       ctypes.byref(g.c), F16) > 0
    # spherical forwards: no split BF16; split FP16 up to 448 theta nodes
    ob_ = api.make_optics(W.optics_gibson_lanni(0.0), _lib.PSF_PROJECT_AXISYMMETRIC)
    bsize = lambda nt, p: cpu_lib.psf_bessel_workspace_size(ctypes.byref(ob_), 4, 16, nt, 64,
                                                            16, 16, p)
    assert bsize(448, F16) > 0 and bsize(200, _lib.PSF_PREC_FP32) > 0
    assert bsize(200, B16) == 0 and b"BF16" in cpu_lib.psf_last_error()
    assert bsize(600, F16) == 0 and b"448" in cpu_lib.psf_last_error()
    assert bsize(200, _lib.PSF_PREC_AUTO) == bsize(200, F16)
    assert bsize(600, _lib.PSF_PREC_AUTO) == bsize(600, _lib.PSF_PREC_FP32)
    hsize = lambda nt, p: cpu_lib.psf_bessel_harmonic_workspace_size(
        ctypes.byref(ob_), 4, 16, nt, 64, 16, 16, 12, p)
    assert hsize(448, F16) > 0 and hsize(600, F16) == 0
    assert hsize(600, _lib.PSF_PREC_AUTO) == hsize(600, _lib.PSF_PREC_FP32)
    # the Bessel adjoint keeps split BF16
    assert cpu_lib.psf_bessel_backward_workspace_size(ctypes.byref(ob_), 4, 16, 200, 64, 16,
                                                      16, B16) > 0


def test_fresnel_bessel_workspaces(cpu_lib):
    """Complex angular weights (Fresnel) are accepted by every Bessel mode and
    the adjoint; the split forward then holds one F plane per order (three
    times the operand rows) and the adjoint the complex J_n operand."""
    plain = W.optics_gibson_lanni(0.0)
    fr = dict(plain, fresnel=True)
    args = (4, 500, 200, 256, 64, 64)
    ws = {}
    for name, d in (("plain", plain), ("fresnel", fr)):
        o = api.make_optics(d, _lib.PSF_PROJECT_AXISYMMETRIC)
        for p in (_lib.PSF_PREC_FP32, _lib.PSF_PREC_SPLIT_FP16):
            ws[name, p, "fwd"] = cpu_lib.psf_bessel_workspace_size(ctypes.byref(o), *args, p)
        for p in (_lib.PSF_PREC_FP32, _lib.PSF_PREC_SPLIT_FP16, _lib.PSF_PREC_SPLIT_BF16):
            ws[name, p, "bwd"] = cpu_lib.psf_bessel_backward_workspace_size(
                ctypes.byref(o), *args, p)
    assert all(v > 0 for v in ws.values()), ws
    F16 = _lib.PSF_PREC_SPLIT_FP16
    # F: 2 x (2 n_slices Kp) 16-bit parts more per extra order
    extra = 2 * 2 * (2 * 500 * 200 * 2)
    assert ws["fresnel", F16, "fwd"] - ws["plain", F16, "fwd"] >= extra
    assert ws["fresnel", _lib.PSF_PREC_FP32, "fwd"] == ws["plain", _lib.PSF_PREC_FP32, "fwd"]
