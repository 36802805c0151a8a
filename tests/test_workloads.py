"""The seeded synthetic inputs follow their stated recipe (CPU): shapes, dtypes, the
deterministic part of each seed (the lamellar cosine, the gyroid level set, the
homogeneous complex Langevin start) and the statistics of the i.i.d. normal part, and the
batch's distribution of grids, contour lengths, field kinds and parameters."""
import numpy as np
import pytest

from paper_1204_5434_gb300 import workloads as wl


def _coords(w):
    return [np.arange(w.n[a]) * (w.L[a] / w.n[a]) for a in range(3)]


def _normal_ok(r, std):
    # sample mean and standard deviation of N i.i.d. normals, 6 standard errors
    N = r.size
    assert abs(r.mean()) <= 6 * std / np.sqrt(N)
    assert abs(r.std() - std) <= 6 * std / np.sqrt(2 * N)


def test_fields_are_deterministic_per_seed():
    a = wl.fields(wl.LAM32)
    b = wl.fields(wl.LAM32)
    c = wl.fields(wl.LAM32.with_(seed=2))
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[1], c[1])


def test_lamellar_seed():
    w = wl.LAM32
    wp, wm = wl.fields(w)
    assert wp.dtype == np.float64 and wp.shape == w.n and np.all(wp == 0.0)
    x = _coords(w)[0]
    _normal_ok(wm - (5.0 * np.cos(2 * np.pi * x / w.L[0]))[:, None, None], 0.1)


def test_gyroid_seed():
    w = wl.GYR64
    wp, wm = wl.fields(w)
    x, y, z = _coords(w)
    X = (2 * np.pi * x / w.L[0])[:, None, None]
    Y = (2 * np.pi * y / w.L[1])[None, :, None]
    Z = (2 * np.pi * z / w.L[2])[None, None, :]
    G = np.sin(X) * np.cos(Y) + np.sin(Y) * np.cos(Z) + np.sin(Z) * np.cos(X)
    _normal_ok(wm - 4.0 * G, 0.1)
    _normal_ok(wp, 0.1)
    assert wl.GYR128.n == (128, 128, 128) and wl.GYR128.Ns == 100 and wl.GYR128.fA == 0.35


def test_homogeneous_complex_langevin_start():
    w = wl.CL64
    wp, wm = wl.fields(w)
    assert wp.dtype == np.complex128 and wm.dtype == np.complex128
    assert np.all(wp.imag == 0.0) and np.all(wm.imag == 0.0)
    _normal_ok(wp.real, 0.05)
    _normal_ok(wm.real - w.chiN * (2 * w.fA - 1) / 2, 0.05)
    assert w.chiN * (2 * w.fA - 1) / 2 == pytest.approx(-4.0)
    assert (w.dt, w.C, w.Ns, w.steps) == (0.01, 50.0, 100, 1000)


def test_large_complex_langevin_parameters():
    w = wl.CL256
    assert w.n == (256, 256, 256) and w.L == (16.0, 16.0, 16.0)
    assert (w.Ns, w.fA, w.chiN, w.C, w.dt, w.steps) == (200, 0.5, 14.0, 100.0, 0.005, 200)


def test_batch_distribution():
    inst = wl.batch_instances()
    assert len(inst) == 256
    assert {w.n[0] for w in inst} == {32, 48, 64} and all(w.n[0] == w.n[1] == w.n[2] for w in inst)
    assert {w.Ns for w in inst} == {50, 100, 200}
    assert all(w.L[0] == w.n[0] / 8.0 for w in inst)
    assert all(0.25 <= w.fA <= 0.5 and 12.0 <= w.chiN <= 25.0 for w in inst)
    assert [w.kind for w in inst] == [wl.SCFT] * 128 + [wl.CL] * 128
    assert len({w.seed for w in inst}) == 256
    wp, wm = wl.sinusoid_fields(inst[0])
    _normal_ok(wp, 0.1)
    # four low-k sinusoids with amplitudes below 2: |W- - noise| <= 8
    assert np.max(np.abs(wm)) <= 8.0 + 6 * 0.1
