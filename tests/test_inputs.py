"""The seeded input recipes (synth.py) have the properties the workloads are stated to
have: the generator is the published SplitMix64, the maps and streams follow their
recipes, and everything is reproducible.  CPU only."""
import numpy as np

from paper_2010_06697_gb300 import synth


def test_mixer_is_the_published_splitmix64():
    """SplitMix64 from state 0: the first output is mix(gamma) = 0xE220A8397B1DCDAF, the
    second mix(2 gamma) = 0x6E789E6AA1B965F4 (the generator's published reference values)."""
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        out = synth._mix64(np.array([g, g * np.uint64(2)], dtype=np.uint64))
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_uniform_and_normal_streams():
    u = synth.uniform(7, 3, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1 / 12) < 2e-3
    assert np.array_equal(u[1000:1010], synth.uniform(7, 3, 10, start=1000))   # counter-based
    assert not np.array_equal(u[:10], synth.uniform(7, 4, 10))                   # tags separate
    z = synth.normal(7, 3, 200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2


def test_inclusion_map_recipe():
    """Stiff spheres of radius 6 voxels added until the inclusion fraction reaches 20 %
    (the last sphere overshoots by less than one sphere's volume); bit-reproducible."""
    ph = synth.inclusion_phase(128, 3, 0)
    assert ph.dtype == np.uint8 and set(np.unique(ph)) == {0, 1}
    frac = ph.mean()
    ball = 4.0 / 3.0 * np.pi * 6.5 ** 3 / 128 ** 3
    assert 0.20 <= frac < 0.20 + ball
    assert np.array_equal(ph, synth.inclusion_phase(128, 3, 0))
    ph2 = synth.inclusion_phase(64, 2, 3, radius=4)
    assert 0.20 <= ph2.mean() < 0.20 + np.pi * 4.5 ** 2 / 64 ** 2


def test_laminate_and_disc_maps():
    ph = synth.laminate_phase(32, 3)
    assert ph.mean() == 0.5
    assert np.array_equal(ph, np.broadcast_to(ph[0, 0], ph.shape))  # depends on x only
    assert ph[0, 0, 15] == 0 and ph[0, 0, 16] == 1
    d = synth.disc_phase(64, 2, 0.25)
    assert abs(d.mean() - np.pi * 0.25 ** 2) < 0.01 and d[32, 32] == 1 and d[0, 0] == 0


def test_director_field_recipe():
    """Unit directors, correlated over about the smoothing length: neighbours are nearly
    parallel, voxels half a cell apart are not."""
    n0 = synth.director_grf(32, 1, corr=4.0)
    assert n0.shape == (3, 32, 32, 32)
    assert np.max(np.abs(np.sum(n0 * n0, axis=0) - 1.0)) < 1e-12
    near = np.mean(np.abs(np.sum(n0 * np.roll(n0, 1, axis=3), axis=0)))
    far = np.mean(np.abs(np.sum(n0 * np.roll(n0, 16, axis=3), axis=0)))
    assert near > 0.95 and far < 0.8


def test_strain_batch_and_serving_recipes():
    F = synth.random_fbar(5, 43)
    assert np.array_equal(F, F.T) and np.max(np.abs(F - np.eye(3))) <= 0.1
    assert synth.smooth_sizes(32, 256) == [32, 36, 48, 54, 64, 72, 96, 108, 128, 144, 162, 192, 216, 256]
    spec = synth.batch_spec(64, 0)
    assert all(s["n"] in synth.BATCH_SIZES for s in spec)
    assert all((s["kind"] == "laminate") == (s["seed"] % 2 == 0) for s in spec)
    reqs = synth.serving_stream(4000, 0, rate_hz=200.0)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0) and abs(np.mean(np.diff(t)) - 1 / 200.0) < 0.05 / 200.0
    sizes = set(synth.smooth_sizes(32, 256))
    assert all(r["n"] in sizes for r in reqs)
    kinds = [r["kind"] for r in reqs]
    for k, p in (("laminate", 0.4), ("inclusion", 0.4), ("lce", 0.2)):
        assert abs(kinds.count(k) / len(kinds) - p) < 0.03
    logn = np.log([r["n"] for r in reqs])
    assert abs(np.mean(logn) - 0.5 * (np.log(32) + np.log(256))) < 0.05   # log-uniform sizes


def test_stored_oracle_solve_matches_todays_inputs():
    """The stored 128^3 oracle solve was made from the inclusion recipe; the recipe still
    produces the same cell (its inclusion fraction and volume-average shear modulus), so the
    GPU test that compares against it compares like with like."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "inclusions128.json")))
    rcp = g["recipe"]
    ph = synth.inclusion_phase(rcp["n"], rcp["dim"], rcp["seed"])
    assert ph.mean() == g["phase_fraction"]
    mu = np.asarray(rcp["mu"])[ph.ravel()]
    assert abs(mu.mean() - g["mu_ref"]) <= 1e-12 * g["mu_ref"]
    assert g["converged"] and np.asarray(g["stress"]).shape == (3, 3)
