"""Pins of the CPU FP64 oracle against what the paper and the mathematics fix (no GPU).

Each pin checks the oracle against something other than itself: the constrained least-squares
definition solved by brute force, the paper's printed stencil, real-space central differences,
hand-derived worked examples (tests/golden), closed forms, invariants, an independent library
FFT.  ``test_planted_mistakes_are_caught`` plants plausible mistakes in a copy of the projector
and checks that the pins reject them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle.projection import VOIGT_IJ, to_tensor, to_voigt, project_spectrum
from fieldgen import gaussian_array, voronoi_stress_field, periodic_voronoi_map

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
OPS = ("ddo", "cdo")


def _load_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _rel(a, b):
    return float(np.sqrt(oracle.frob2(a - b).sum() / max(oracle.frob2(b).sum(), 1e-300)))


# ---------------------------------------------------------------- transforms (Sec. 4)

def test_transforms_agree_with_each_other_and_numpy():
    x = gaussian_array((6, 3, 4, 5), 11) + 1j * gaussian_array((6, 3, 4, 5), 12)
    ref = np.fft.fftn(x, axes=(-3, -2, -1))
    for f in (oracle.dft3_naive, oracle.dft3_direct, oracle.fft3):
        y = f(x)
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    back = oracle.dft3_direct(oracle.dft3_direct(x), inverse=True)
    assert np.abs(back - x).max() < 1e-13
    back = oracle.dft3_naive(oracle.dft3_naive(x), inverse=True)
    assert np.abs(back - x).max() < 1e-13
    # Parseval: sum |x|^2 = sum |X|^2 / N
    assert abs((np.abs(x) ** 2).sum() - (np.abs(ref) ** 2).sum() / 60) < 1e-10


def test_direct_dft_matches_numpy_on_prime_and_odd_sizes():
    for n in (7, 9, 11, 13, 97):
        x = gaussian_array((2, n), n)
        y = oracle.dft_axis_direct(x, -1)
        ref = np.fft.fft(x, axis=-1)
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------- operators (Sec. 4.1, 4.2)

def test_wavevector_golden_n8():
    rows = _load_rows("wavevector_n8.txt")
    cdo = np.array([float(r[1]) for r in rows])
    ddo = np.array([float(r[2]) for r in rows])
    assert np.allclose(oracle.wavevector(8, 1.0, "cdo"), cdo, rtol=0, atol=1e-15)
    assert np.allclose(oracle.wavevector(8, 1.0, "ddo"), ddo, rtol=0, atol=1e-15)
    # spacing scales 1/h; odd N has no Nyquist zero
    assert np.allclose(oracle.wavevector(8, 2.0, "cdo"), cdo / 2.0, atol=1e-15)
    assert np.all(oracle.wavevector(7, 1.0, "cdo")[1:] != 0.0)


def test_cdo_derivative_of_trig_polynomial_is_exact():
    n, h = 12, 0.5
    x = (np.arange(n) * h)[None, None, None, :]
    L = n * h
    f = np.zeros((6, 1, 1, n))
    want = np.zeros_like(f)
    for m in range(1, n // 2):       # below Nyquist: the spectral derivative is exact
        f[0] += np.sin(2 * np.pi * m * x[0] / L) * (m + 1)
        want[0] += (2 * np.pi * m / L) * np.cos(2 * np.pi * m * x[0] / L) * (m + 1)
    # (div S)_0 = d_x S_xx when only S_xx is non-zero
    d = oracle.divergence(f, "cdo", (h, 1.0, 1.0))
    assert np.abs(d[0] - want[0]).max() < 1e-11
    assert np.abs(d[1:]).max() < 1e-12


def test_ddo_spectral_divergence_equals_central_differences():
    s = gaussian_array((6, 6, 5, 7), 3)
    h = (1.0, 0.8, 1.7)
    a = oracle.divergence(s, "ddo", h)
    b = oracle.divergence_central_diff(s, h)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_stencil_is_the_printed_one_and_its_symbol_is_ddo_k_to_the_4():
    rows = _load_rows("stencil25_sec4_2.txt")
    golden = {(int(r[0]), int(r[1]), int(r[2])): float(r[3]) for r in rows}
    assert golden == oracle.operators.paper_stencil_weights()
    shape, h = (8, 10, 12), 0.7
    f = gaussian_array(shape, 5)
    real_space = oracle.stencil25_apply(f, h, golden)
    via_paper_symbol = np.real(oracle.ifft3(oracle.biharmonic_symbol_paper(shape, h)
                                            * oracle.fft3(f)))
    xi = oracle.wavevector_grids(shape, (h, h, h), "ddo")
    k4 = (xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2) ** 2
    via_k4 = np.real(oracle.ifft3(k4 * oracle.fft3(f)))
    scale = np.abs(real_space).max()
    assert np.abs(real_space - via_paper_symbol).max() < 1e-12 * scale
    assert np.abs(real_space - via_k4).max() < 1e-12 * scale


# ---------------------------------------------------------------- the definition (Sec. 3.2)

@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("shape,h", [((4, 4, 4), (1.0, 1.0, 1.0)),
                                     ((3, 4, 5), (1.0, 1.3, 0.7)),
                                     ((2, 6, 4), (0.5, 1.0, 2.0)),
                                     ((5, 3, 7), (1.0, 1.0, 1.0))])
def test_projection_is_the_constrained_least_squares_minimiser(op, shape, h):
    s = gaussian_array((6,) + shape, sum(shape)) + 3.0
    brute = oracle.project_bruteforce(s, op, h)
    for tr in ("fft", "direct"):
        got = oracle.project(s, op, h, transform=tr)
        assert _rel(got, brute) < 1e-12
    if np.prod(shape) <= 4096:
        assert _rel(oracle.project(s, op, h, transform="naive"), brute) < 1e-12


def test_plane_wave_golden_examples():
    rows = _load_rows("plane_wave_4cube.txt")
    a = np.array([[1.0, 2, 3], [2, 4, 5], [3, 5, 6]])
    z, y, x = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
    for r in rows:
        if r[0] == "NORMS2":
            continue
        m = [int(v) for v in r[:3]]
        want6 = np.array([float(v) for v in r[3:9]])
        c = np.cos(2 * np.pi * (m[0] * x + m[1] * y + m[2] * z) / 4)
        s = to_voigt(a[:, :, None, None, None] * c[None, None])
        out = oracle.project(s, "ddo")
        assert np.abs(out - want6[:, None, None, None] * c[None]).max() < 1e-13
        if m == [1, 1, 0]:
            nrm = [float(v) for v in [q for q in rows if q[0] == "NORMS2"][0][1:]]
            got = oracle.norms(s, out, "ddo")
            keys = ("norm_in", "norm_out", "resid_l2", "resid_linf", "div_in_l2", "div_out_l2")
            for k, w2 in zip(keys, nrm):
                assert abs(got[k] - math.sqrt(w2)) < 1e-12, k


def test_constant_field_unchanged_and_laminate_closed_form():
    c = np.arange(1.0, 7.0)
    s = np.broadcast_to(c[:, None, None, None], (6, 4, 5, 6)).copy()
    for op in OPS:
        assert np.abs(oracle.project(s, op) - s).max() < 1e-13
    # laminate: S depends on x only (odd nx, so no Nyquist mode).  Traction continuity across
    # the layers: xx, xz, xy become their means; yy, zz, yz are untouched.
    nx = 9
    prof = gaussian_array((6, 1, 1, nx), 8)
    s = np.broadcast_to(prof, (6, 3, 4, nx)).copy()
    for op in OPS:
        out = oracle.project(s, op, (0.7, 1.0, 1.2))
        for comp in (0, 4, 5):
            assert np.abs(out[comp] - s[comp].mean()).max() < 1e-13
        for comp in (1, 2, 3):
            assert np.abs(out[comp] - s[comp]).max() < 1e-13


@pytest.mark.parametrize("op", OPS)
def test_projector_invariants(op):
    shape, h = (8, 6, 10), (1.0, 1.2, 0.9)
    a = voronoi_stress_field(shape, 6, 100.0, 10.0, 101).numpy()
    b = gaussian_array((6,) + shape, 102)
    pa, pb = oracle.project(a, op, h), oracle.project(b, op, h)
    scale = oracle.inner(a, a)
    assert _rel(oracle.project(pa, op, h), pa) < 1e-13                           # P^2 = P
    assert abs(oracle.inner(pa, b) - oracle.inner(a, pb)) < 1e-12 * math.sqrt(
        scale * oracle.inner(b, b))                                              # self-adjoint
    assert abs(oracle.inner(a - pa, pa)) < 1e-12 * scale                          # orthogonal
    assert abs(oracle.inner(a, a) - oracle.inner(pa, pa) - oracle.inner(a - pa, a - pa)) \
        < 1e-12 * scale                                                           # Pythagoras
    p_ab = oracle.project(a + 2.5 * b, op, h)
    assert _rel(p_ab, pa + 2.5 * pb) < 1e-13                                      # linear
    d = oracle.divergence(pa, op, h)
    assert np.abs(d).max() < 1e-12 * np.abs(oracle.divergence(a, op, h)).max()


def test_ddo_projection_is_divergence_free_by_central_differences():
    shape, h = (6, 8, 10), (1.0, 0.5, 1.5)
    s = voronoi_stress_field(shape, 5, 100.0, 10.0, 7).numpy()
    out = oracle.project(s, "ddo", h)
    d = oracle.divergence_central_diff(out, h)
    d0 = oracle.divergence_central_diff(s, h)
    assert np.abs(d).max() < 1e-12 * np.abs(d0).max()


@pytest.mark.parametrize("op", OPS)
def test_equilibrated_field_unchanged_and_symgrad_reduced_to_mean(op):
    shape, h = (6, 8, 10), (1.0, 1.1, 0.9)
    hpot = gaussian_array((6,) + shape, 21)
    truth = oracle.beltrami_field(hpot, h, op)
    c = np.array([5.0, -3.0, 2.0, 1.0, 0.5, -1.0])[:, None, None, None]
    assert np.abs(oracle.divergence(truth, op, h)).max() < 1e-11 * np.abs(truth).max()
    out = oracle.project(truth + c, op, h)
    assert _rel(out, truth + c) < 1e-12
    vec = gaussian_array((3,) + shape, 22)
    sg = oracle.symgrad_field(vec, h, op)
    out = oracle.project(sg + c, op, h)
    assert np.abs(out - c).max() < 1e-12 * np.abs(sg).max()
    # recovery of the truth from truth + symmetric-gradient perturbation (Sec. 5.1, Fig. 3a,b)
    out = oracle.project(truth + sg, op, h)
    assert _rel(out, truth) < 1e-12


@pytest.mark.parametrize("op", OPS)
def test_literal_euler_lagrange_route_equals_closed_form(op):
    for shape, h in (((6, 8, 4), (1.0, 1.0, 1.0)), ((5, 6, 7), (1.0, 1.3, 0.8))):
        s = gaussian_array((6,) + shape, 31)
        lit = oracle.project_literal(s, op, h)
        assert _rel(lit, oracle.project(s, op, h, nyq="zero")) < 1e-12
        keep = oracle.project(s, op, h, nyq="keep")
        if all(n % 2 == 1 for n in shape):
            # odd sizes have no Nyquist corners: both policies coincide
            assert _rel(lit, keep) < 1e-12


def test_keep_and_zero_differ_only_at_degenerate_modes():
    shape = (4, 6, 8)
    s = gaussian_array((6,) + shape, 41)
    diff = oracle.fft3(oracle.project(s, "ddo") - oracle.project(s, "ddo", nyq="zero"))
    mask = np.zeros(shape, dtype=bool)
    for kz in (0, 2):
        for ky in (0, 3):
            for kx in (0, 4):
                mask[kz, ky, kx] = True
    mask[0, 0, 0] = False
    assert np.abs(diff[:, ~mask]).max() < 1e-10
    assert np.abs(diff[:, mask]).max() > 1e-3


def test_recovery_error_equals_projection_of_perturbation():
    # Sec. 5.1: P(truth + delta) - truth = P(delta) for an equilibrated truth
    shape = (8, 8, 8)
    truth = oracle.beltrami_field(gaussian_array((6,) + shape, 51), op="ddo")
    delta = voronoi_stress_field(shape, 10, 50.0, 0.0, 52).numpy()
    lhs = oracle.project(truth + delta, "ddo") - truth
    assert _rel(lhs, oracle.project(delta, "ddo")) < 1e-12


def test_norms_definitions():
    shape = (6, 8, 10)
    s = voronoi_stress_field(shape, 5, 100.0, 10.0, 61).numpy()
    out = oracle.project(s, "ddo")
    n = oracle.norms(s, out, "ddo")
    assert abs(n["norm_in"] ** 2 - n["norm_out"] ** 2 - n["resid_l2"] ** 2) < 1e-10 * n["norm_in"] ** 2
    assert n["div_out_l2"] < 1e-12 * n["div_in_l2"]
    assert np.allclose(n["mean"], s.mean(axis=(1, 2, 3)))
    assert n["resid_linf"] == pytest.approx(np.abs(s - out).max())
    d = oracle.divergence_central_diff(s)
    assert n["div_in_l2"] == pytest.approx(math.sqrt((d ** 2).sum(0).mean()), rel=1e-12)


# ---------------------------------------------------------------- pins reject planted mistakes

def _mutant(kind):
    def proj(s6, h=(1.0, 1.0, 1.0)):
        shape = s6.shape[1:]
        c0 = s6.mean(axis=(1, 2, 3))
        t = to_tensor(oracle.fft3(s6 - c0[:, None, None, None]))
        xi = [np.broadcast_to(a, shape) for a in oracle.wavevector_grids(shape, h, "ddo")]
        if kind == "swapped_axes":
            xi = [xi[2], xi[1], xi[0]]
        k2 = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
        deg = k2 == 0
        n = np.stack([a / np.sqrt(np.where(deg, 1.0, k2)) for a in xi])
        v = np.einsum("ij...,j...->i...", t, n)
        sc = np.einsum("i...,i...->...", n, v)
        sign = -1.0 if kind == "sign" else 1.0
        last = 0.0 if kind == "dropped_term" else 1.0
        out = t - n[:, None] * v[None, :] - sign * v[:, None] * n[None, :] \
            + last * sc * n[:, None] * n[None, :]
        out = np.where(deg[None, None], t, out)
        return np.real(oracle.ifft3(to_voigt(out))) + c0[:, None, None, None]
    return proj


def test_planted_mistakes_are_caught():
    shape = (4, 4, 6)
    s = gaussian_array((6,) + shape, 71)
    brute = oracle.project_bruteforce(s, "ddo")
    assert _rel(_mutant("none")(s), brute) < 1e-12
    for kind in ("sign", "dropped_term", "swapped_axes"):
        assert _rel(_mutant(kind)(s), brute) > 1e-3, kind


# ---------------------------------------------------------------- generator recipe

def test_voronoi_map_is_periodic_nearest_seed():
    shape, g, seed = (5, 6, 7), 9, 3
    gm = periodic_voronoi_map(shape, g, seed).numpy()
    from fieldgen import _grain_seeds
    seeds = _grain_seeds(shape, g, seed)
    nz, ny, nx = shape
    box = np.array([nx, ny, nz], float)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                p = np.array([x + 0.5, y + 0.5, z + 0.5])
                d = seeds - p
                d -= box * np.round(d / box)
                dist = np.sqrt((d ** 2).sum(1))
                best = np.flatnonzero(dist <= dist.min() * (1 + 1e-6))
                assert gm[z, y, x] in best


@pytest.mark.parametrize("slab", [1, 3, 7])
def test_large_grid_projection_and_norms_equal_the_whole_field_ones(slab):
    """project_large / norms_large (component-at-a-time transforms, projector on z-slabs) give the
    pinned whole-field project / norms: the same per-mode arithmetic, grouped differently."""
    s = voronoi_stress_field((10, 12, 8), 5, 100.0, 10.0, 31).numpy()
    for op in ("ddo", "cdo"):
        for nyq in ("keep", "zero"):
            h = (1.0, 0.7, 1.2)
            a = oracle.project(s, op, h, nyq)
            b = oracle.project_large(s.astype(np.float32), op, h, nyq, slab=slab)
            a32 = oracle.project(s.astype(np.float32).astype(np.float64), op, h, nyq)
            assert np.abs(b - a32).max() <= 1e-13 * np.abs(a32).max(), (op, nyq)
            assert np.abs(oracle.project_large(s, op, h, nyq, slab=slab) - a).max() <= \
                1e-13 * np.abs(a).max()
            n1 = oracle.norms(s, a, op, h)
            n2 = oracle.norms_large(s, a, op, h)
            for k in n1:
                assert np.allclose(n2[k], n1[k], rtol=1e-12, atol=1e-14 * n1["norm_in"]), (k, op)
