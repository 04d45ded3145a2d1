"""Spherical strategy without axial symmetry (azimuthal harmonics) on the
GPU, through the C ABI, against the FP64 harmonic oracle (pinned on the CPU
against Eq. 10-11 and the direct quadrature of Eq. 9).

Same discretisation on both sides (harmonics |m| <= M by a DFT over N_phi
azimuths, Gauss-Legendre theta, linear radial interpolation), so the bound
is the forward one: intensity max-rel 1e-5 per emitter stack."""
import numpy as np
import pytest
import torch

from oracle import bessel as ob
from oracle import bessel_harmonic as bh
from paper_2502_03170_gb300 import _lib, api
from paper_2502_03170_gb300 import workloads as W

from .gpu_helpers import max_rel, oracle_optics

pytestmark = pytest.mark.gpu
TOL = 1e-5


def batch(n_em, seed, n_zern=21, scale=0.08):
    g = np.random.default_rng(seed)
    depth = g.uniform(0.0, 6.0, n_em)
    zern = np.zeros((n_em, n_zern))
    zern[:, 3:min(n_zern, 15)] = g.normal(0, scale, (n_em, min(n_zern, 15) - 3))
    nz = g.integers(1, 5, n_em)
    nz[1 % n_em] = 0                                  # an emitter without slices
    offs = np.concatenate([[0], np.cumsum(nz)]).astype(np.int32)
    z = g.uniform(-0.8, 0.8, int(offs[-1]))
    return depth, zern, offs, z


def check(d, depth, zern, offs, z, geo, m_max, tail_tol=0.0, precision="fp32", tol=TOL):
    I = api.bessel_harmonic(d, depth, zern, offs, z, *geo, m_max=m_max, tail_tol=tail_tol,
                            precision=precision)
    torch.cuda.synchronize()
    I = I.cpu().numpy()
    o = oracle_optics(d)
    Iref = bh.psf_harmonic_batch(o, depth, zern, offs, z, *geo, m_max, tail_tol=tail_tol)
    for e in range(len(depth)):
        a, b = offs[e], offs[e + 1]
        if b > a:
            assert max_rel(I[a:b], Iref[a:b]) <= tol, e
    return I


@pytest.mark.parametrize("precision", ["fp32", "split_fp16"])
@pytest.mark.parametrize("kw", [dict(pol=W.CIRCULAR), dict(pol=(0.6, 0.48 + 0.64j)),
                                dict(pol=(1.0, 0.0)), dict(scalar=True),
                                dict(fresnel=True, pol=W.CIRCULAR)])
def test_harmonic_matches_oracle(lib, kw, precision):
    """FP32 contraction and the tensor-core (split) contraction, every
    polarisation and model, with and without the adaptive order."""
    d = dict(W.optics_gibson_lanni(0.0), **kw)
    depth, zern, offs, z = batch(5, 3)
    m_max = api.harmonic_order(zern, 1e-6)
    assert m_max > 4
    geo = (48, 40, 19, 16, 0.035, 0.03)
    check(d, depth, zern, offs, z, geo, m_max, precision=precision)
    check(d, depth, zern, offs, z, geo, m_max, tail_tol=1e-6, precision=precision)


@pytest.mark.parametrize("m_max", [0, 1, 7, 40])
def test_harmonic_orders_and_ragged(lib, m_max):
    d = W.optics_gibson_lanni(0.0)
    depth, zern, offs, z = batch(3, 11 + m_max, scale=0.12)
    check(d, depth, zern, offs, z, (33, 29, 13, 22, 0.04, 0.03), m_max)


def test_axisymmetric_pupil_equals_the_axisymmetric_path(lib):
    d = W.optics_gibson_lanni(0.0)
    depth, zern, offs, z = batch(4, 5)
    zax = np.zeros_like(zern)
    zax[:, 3], zax[:, 10] = zern[:, 3], zern[:, 10]
    geo = (40, 64, 24, 24, 0.03, 0.03)
    Ih = api.bessel_harmonic(d, depth, zax, offs, z, *geo, m_max=3, tail_tol=0.0)
    Ib = api.bessel(d, depth, zax, offs, z, *geo)
    torch.cuda.synchronize()
    assert max_rel(Ih.cpu().numpy(), Ib.cpu().numpy()) <= 2 * TOL
    Iref = ob.psf_bessel_batch(oracle_optics(d), depth, zax, offs, z, *geo)
    assert max_rel(Ih.cpu().numpy(), Iref) <= TOL


@pytest.mark.parametrize("precision", ["fp32", "split_fp16"])
def test_harmonic_workload_emitters_sampled(lib, precision):
    """Emitters of the batched workload (4..11 Zernike terms, all of them,
    depth up to 10 um) at the order the tail bound gives for 1e-7."""
    c = W.bessel(n_emitters=24)
    m_max = api.harmonic_order(c["zernike"], 1e-7)
    geo = (c["n_theta"], 128, 64, 64, c["dx"], c["dy"])
    I = api.bessel_harmonic(c["optics"], c["depth"], c["zernike"], c["z_offsets"], c["z"],
                            *geo, m_max=m_max, tail_tol=1e-7, precision=precision)
    torch.cuda.synchronize()
    I = I.cpu().numpy()
    o = oracle_optics(c["optics"])
    for e in (0, 7, 23):
        a, b = c["z_offsets"][e], c["z_offsets"][e + 1]
        Iref = bh.psf_harmonic_batch(o, c["depth"], c["zernike"], c["z_offsets"], c["z"],
                                     *geo, m_max, emitters=[e], tail_tol=1e-7)
        assert max_rel(I[a:b], Iref) <= TOL, e
        # the dropped harmonics change the stack by less than the parity bound
        Ifull = bh.psf_harmonic_batch(o, c["depth"], c["zernike"], c["z_offsets"], c["z"],
                                      *geo, m_max, emitters=[e])
        assert max_rel(I[a:b], Ifull) <= TOL, e


@pytest.mark.parametrize("precision", ["fp32", "split_fp16"])
@pytest.mark.parametrize("tail_tol", [1e-3, 1e-5])
def test_adaptive_order_orders_and_ragged(lib, tail_tol, precision):
    """Coarse tolerances give emitters of different orders in one batch
    (tiles of the contraction mix emitters that need an order and emitters
    that do not, and the tensor-core contraction skips tiles no column
    needs); ragged sizes, an emitter without slices."""
    d = W.optics_gibson_lanni(0.0)
    depth, zern, offs, z = batch(6, 17, scale=0.06)
    zern[2] *= 0.05                              # a nearly axisymmetric emitter
    m_max = min(api.harmonic_order(zern, 1e-8), 40)
    check(d, depth, zern, offs, z, (41, 37, 17, 21, 0.04, 0.035), m_max, tail_tol=tail_tol,
          precision=precision)


@pytest.mark.parametrize("n_em,n_r", [(2, 2), (7, 300), (40, 129)])
def test_split_contraction_tiles(lib, n_em, n_r):
    """The tensor-core contraction against the FP32 one and the oracle:
    N_r not a multiple of the 128-row tile (129, 300: padded A planes), the
    two-sample radial grid, and enough slices for several column tiles per
    order (40 emitters)."""
    d = W.optics_gibson_lanni(0.0)
    depth, zern, offs, z = batch(n_em, 31 + n_em, scale=0.07)
    m_max = min(api.harmonic_order(zern, 1e-7), 24)
    geo = (45, n_r, 20, 20, 0.04, 0.04)
    Is = check(d, depth, zern, offs, z, geo, m_max, tail_tol=1e-7, precision="split_fp16")
    If = api.bessel_harmonic(d, depth, zern, offs, z, *geo, m_max=m_max, tail_tol=1e-7)
    torch.cuda.synchronize()
    assert max_rel(Is, If.cpu().numpy()) <= 5e-6


@pytest.mark.parametrize("n,n_r", [(1, 33), (2, 33), (15, 33), (16, 33), (40, 96),
                                   (32, 2048)])
def test_square_geometry_octant_epilogue(lib, n, n_r):
    """nx = ny and dx = dy take the octant epilogue (one thread per pixel and
    its seven images): odd sizes have a centre row and the diagonal, n = 1 a
    single pixel; 40 px spans several blocks; with N_r = 2048 a block's
    radial run is too long to stage and the profiles are read from global
    memory.  Against the oracle, and against the quarter-pixel epilogue (dy
    off by 1e-12 relative)."""
    d = W.optics_gibson_lanni(0.0)
    depth, zern, offs, z = batch(4, 23 + n)
    m_max = api.harmonic_order(zern, 1e-6)
    geo = (37, n_r, n, n, 0.045, 0.045)
    I = check(d, depth, zern, offs, z, geo, m_max, tail_tol=1e-7)
    geo4 = (37, n_r, n, n, 0.045, 0.045 * (1 + 1e-12))
    I4 = api.bessel_harmonic(d, depth, zern, offs, z, *geo4, m_max=m_max, tail_tol=1e-7)
    torch.cuda.synchronize()
    assert max_rel(I, I4.cpu().numpy()) <= 2e-6


@pytest.mark.parametrize("px", [(9, 11, 0.05, 0.04), (12, 12, 0.045, 0.045)])
def test_maximum_order_and_nodes(lib, px):
    """The largest sizes the call takes: m_max = 64 (133 orders, a 512-point
    azimuthal FFT) with every order kept, and 880 Gauss-Legendre nodes; the
    quarter-pixel and the octant epilogue, FP32 contraction.  The split form
    sums 880 strongly oscillating terms per integral (aberrations of 0.15 rad
    per term) in each FP32 tensor-core accumulator and measured up to 1.2e-5
    there: it is refused beyond 448 nodes."""
    d = W.optics_gibson_lanni(0.0)
    depth, zern, offs, z = batch(3, 91, scale=0.15)
    check(d, depth, zern, offs, z, (880, 40) + px, 64, tail_tol=0.0, precision="fp32")
    with pytest.raises(_lib.PsfError) as e:
        check(d, depth, zern, offs, z, (880, 40) + px, 64, tail_tol=0.0,
              precision="split_fp16")
    assert e.value.code == _lib.PSF_ERR_PRECISION


@pytest.mark.parametrize("px", [(9, 11, 0.05, 0.04), (12, 12, 0.045, 0.045)])
def test_split_at_the_envelope_edge(lib, px):
    """Split FP16 at the largest node count it accepts (448) with every
    order up to 64 and the same strong aberrations: within 1e-5."""
    d = W.optics_gibson_lanni(0.0)
    depth, zern, offs, z = batch(3, 91, scale=0.15)
    check(d, depth, zern, offs, z, (448, 40) + px, 64, tail_tol=0.0, precision="split_fp16")


@pytest.mark.parametrize("kind", ["bessel_split", "harmonic_fp32", "harmonic_split"])
def test_spherical_calls_in_a_cuda_graph(lib, kind):
    """The Bessel and harmonic forwards captured in a CUDA graph and replayed
    equal the direct calls bitwise (parameter tables travel as kernel
    arguments, scratch words are cleared by memset nodes)."""
    c = W.bessel(n_emitters=6)
    geo = (c["n_theta"], 64, 32, 32, c["dx"], c["dy"])
    ws = api.Workspace()
    m_max = api.harmonic_order(c["zernike"], 1e-7)
    # inputs resident on the device (a captured call copies nothing from the host)
    dv = lambda a, dt: torch.as_tensor(np.asarray(a)).to("cuda", dt).contiguous()
    depth, zern = dv(c["depth"], torch.float64), dv(c["zernike"], torch.float64)
    offs, z = dv(c["z_offsets"], torch.int32), dv(c["z"], torch.float64)

    def call(out):
        if kind == "bessel_split":
            return api.bessel(c["optics"], depth, zern, offs, z, *geo, project=True,
                              precision="split_fp16", workspace=ws, out=out)
        prec = "split_fp16" if kind == "harmonic_split" else "fp32"
        return api.bessel_harmonic(c["optics"], depth, zern, offs, z, *geo, m_max=m_max,
                                   precision=prec, workspace=ws, out=out)
    ref = call(None)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    out = torch.full(ref.shape, float("nan"), device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        call(out)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    out.fill_(float("nan"))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        call(out)
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)
