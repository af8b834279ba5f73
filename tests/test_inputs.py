"""The seeded input recipe (inputs/synth.py), on CPU.

The generators stand in for the paper's charged-defect right-hand sides
(Sec. 5.2): Gaussian blobs with minimum-image distances on periodic axes and
clipped windows elsewhere, a grid sum of +-1 per defect in charge mode or a
drawn peak in amplitude mode, optional noise, and the normalisation
||eta||_2 = 1/N of the paper's experiments (eq. normalization).  These tests
pin each part of that recipe, and the workload specifications built on it.
"""
import numpy as np
import pytest

from inputs import synth


def test_storage_order_and_type():
    eta = synth.defect_rhs(12, 10, 6, ("P", "D", "N"), 5, 1.5, seed=3)
    assert eta.shape == (6, 10, 12) and eta.dtype == np.float64 and eta.flags["C_CONTIGUOUS"]


def test_seeded_and_reproducible():
    a = synth.defect_rhs(16, 12, 8, ("P", "P", "N"), 10, (1.0, 4.0), seed=11, noise_std=1e-3)
    b = synth.defect_rhs(16, 12, 8, ("P", "P", "N"), 10, (1.0, 4.0), seed=11, noise_std=1e-3)
    c = synth.defect_rhs(16, 12, 8, ("P", "P", "N"), 10, (1.0, 4.0), seed=12, noise_std=1e-3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


@pytest.mark.parametrize("shape", [(64, 64, 1), (32, 24, 16)])
def test_paper_normalisation(shape):
    nx, ny, nz = shape
    eta = synth.defect_rhs(nx, ny, nz, ("P", "N", "D"), 20, 2.0, seed=5, noise_std=1e-3)
    assert np.linalg.norm(eta.ravel()) == pytest.approx(1.0 / (nx * ny * nz), rel=1e-13)


def test_charge_mode_blob_sums_to_its_charge():
    """Fully periodic grid: the whole blob stays on the grid, so its grid sum is the charge."""
    for q in (1.0, -1.0):
        eta = synth.gaussian_defects((10, 12, 14), (True, True, True), [(3.7, 5.2, 1.1)], [1.5], [q], "charge")
        assert eta.sum() == pytest.approx(q, abs=1e-13)


def test_amplitude_mode_peak_on_a_grid_point():
    eta = synth.gaussian_defects((9, 9, 9), (False, False, False), [(4.0, 4.0, 4.0)], [2.0], [0.7], "amplitude")
    assert eta.max() == pytest.approx(0.7, rel=1e-15)
    assert eta[4, 4, 4] == eta.max()


def test_minimum_image_on_periodic_axes_and_clipping_elsewhere():
    """A blob centred at x = 0: on a periodic axis the value at x = n-1 equals the one at x = 1 (distance 1
    through the wrap); on a Dirichlet axis the window is clipped and nothing appears at x = n-1."""
    n = 16
    per = synth.gaussian_defects((1, 1, n), (True, False, False), [(0.0, 0.0, 0.0)], [1.5], [1.0], "amplitude")
    assert per[0, 0, n - 1] == pytest.approx(per[0, 0, 1], rel=1e-15)
    assert per[0, 0, n - 1] > 0
    clip = synth.gaussian_defects((1, 1, n), (False, False, False), [(0.0, 0.0, 0.0)], [1.5], [1.0], "amplitude")
    assert clip[0, 0, n - 1] == 0.0
    assert clip[0, 0, 1] == pytest.approx(per[0, 0, 1], rel=1e-15)


def test_wide_blob_on_a_short_periodic_axis_folds_every_image():
    """A window wider than the axis folds all images: the profile is then the periodic sum."""
    n, s, c = 4, 3.0, 1.0
    eta = synth.gaussian_defects((1, 1, n), (True, False, False), [(c, 0.0, 0.0)], [s], [1.0], "amplitude")
    half = int(np.ceil(4.0 * s))
    idx = np.arange(int(np.floor(c)) - half, int(np.floor(c)) + half + 2)
    expect = np.zeros(n)
    np.add.at(expect, np.mod(idx, n), np.exp(-0.5 * ((idx - c) / s) ** 2))
    assert np.allclose(eta[0, 0], expect, rtol=1e-15, atol=0)


def test_workloads_follow_their_specifications():
    w = synth.workload_2d_dirichlet()
    assert (w["nx"], w["ny"], w["nz"], w["bcs"], w["tol"]) == (64, 64, 1, ("D", "D", "D"), 1e-12)
    w = synth.workload_film_128()
    assert (w["nx"], w["ny"], w["nz"], w["bcs"], w["tol"]) == (128, 128, 64, ("P", "P", "DN"), 1e-10)
    w = synth.workload_cuboid_256(nz=16)
    assert (w["nx"], w["ny"], w["nz"], w["bcs"]) == (256, 256, 16, ("P", "P", "N"))
    assert np.linalg.norm(w["eta"].ravel()) == pytest.approx(1.0 / (256 * 256 * 16), rel=1e-13)


def test_batched_specs():
    specs = synth.batched_specs()
    assert len(specs) == 48
    for s in specs:
        assert s["nx"] in (64, 96, 128, 160) and s["ny"] in (64, 96, 128, 160) and s["nz"] in (32, 64, 96)
        assert all(b in synth.BC_NAMES for b in s["bcs"])
        assert 1 <= s["nrhs"] <= 8
    assert specs == synth.batched_specs()  # seeded


def test_serving_sessions_move_one_percent_of_their_defects():
    sessions = synth.serving_sessions()
    assert len(sessions) == 16
    for ses in sessions:
        assert ses.nx in range(64, 257, 32) and ses.ny in range(64, 257, 32) and ses.nz in range(32, 193, 32)
    ses = sessions[0]
    before = ses.centres.copy()
    ses.step()
    moved = np.any(ses.centres != before, axis=1)
    assert moved.sum() == max(1, len(ses.charges) // 100)


def test_serving_incremental_update_equals_fresh_field():
    """apply_moves on a field at step k-2 with the moves of steps k-1 and k gives the field of step k (the
    bench's two-buffer scheme), at the scale fixed on the first step."""
    ses = synth.ServingSession(7, 64, 32, 16, ("P", "D", "N"))
    scale = ses.paper_scale()
    periodic = tuple(b == "P" for b in ses.bcs)

    def fresh():
        return scale * synth.gaussian_defects((ses.nz, ses.ny, ses.nx), periodic, ses.centres,
                                              np.full(len(ses.charges), ses.sigma), ses.charges, "charge")

    buf = fresh()
    np.testing.assert_allclose(np.linalg.norm(buf), 1.0 / buf.size, rtol=1e-12)
    m1 = ses.step()
    m2 = ses.step()
    ses.apply_moves(buf, m1, scale)
    ses.apply_moves(buf, m2, scale)
    np.testing.assert_allclose(buf, fresh(), rtol=0, atol=1e-12 * np.abs(buf).max())


def test_poisson_arrivals():
    t = synth.poisson_arrivals(200.0, 20000, seed=1)
    assert np.all(np.diff(t) > 0)
    assert np.array_equal(t, synth.poisson_arrivals(200.0, 20000, seed=1))
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential with mean 5 ms: the sample mean of 20000 gaps is within 4 standard errors
    assert abs(gaps.mean() - 0.005) <= 4 * 0.005 / np.sqrt(len(gaps))
