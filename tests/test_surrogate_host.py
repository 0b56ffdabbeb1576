"""Host side of the MLP surrogate (no GPU): the seeded training links, the
per-channel features and the training envelope that decides between the MLP and
the integrator."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def S():
    from paper_2412_11614_gb300 import _build
    _build.build()  # features use the library's format moments (host code)
    from paper_2412_11614_gb300 import surrogate
    return surrogate


def test_surrogate_links_are_seeded_and_in_range(workloads):
    a, b = workloads.surrogate_link(7), workloads.surrogate_link(7)
    assert a.launch_power_w == b.launch_power_w and a.formats == b.formats and a.notes == b.notes
    for seed in range(1, 200):
        w = workloads.surrogate_link(seed)
        n = w.notes
        assert 1 <= n["n_spans"] <= 30 and 50.0 <= n["length_km"] <= 120.0 and 0.014 <= n["cr"] <= 0.042
        assert -2.0 <= n["p0_dbm"] <= 4.0 and -3.0 <= n["tilt_db"] <= 3.0
        assert len(w.centre_hz) == 120 and len(w.spans) == n["n_spans"]
        assert all(s == w.spans[0] for s in w.spans)


def test_features_shape_and_definitions(S, workloads):
    w = workloads.surrogate_link(3)
    f = S.features(w)
    assert f.shape == (120, S.N_FEAT) and np.all(np.isfinite(f))
    x = f[:, 0]
    assert np.isclose(x[0], -x[-1]) and np.allclose(f[:, 1], x ** 2) and np.allclose(f[:, 2], x ** 3)
    p_dbm = 10 * np.log10(np.asarray(w.launch_power_w) / 1e-3)
    assert np.allclose(f[:, 3], (p_dbm - 1.0) / 3.0)
    assert np.allclose(f[:, 9], (len(w.spans) - 15.5) / 15.0)
    assert np.all(f[:, 17] == 1.0)
    # the interference sums: a channel whose power is raised sees less relative interference
    w2 = workloads.surrogate_link(3)
    w2.launch_power_w = list(w2.launch_power_w)
    w2.launch_power_w[60] *= 4.0
    f2 = S.features(w2)
    assert f2[60, 18] < f[60, 18] and f2[59, 18] > f[59, 18]


def test_envelope(S, workloads):
    w = workloads.surrogate_link(5)
    assert S.in_envelope(w)
    assert not S.in_envelope(workloads.config_small())              # 5 channels
    assert not S.in_envelope(workloads.config_cl(n_spans=40))       # 40 spans
    odd = workloads.surrogate_link(5)
    odd.spans = list(odd.spans)
    odd.spans[0] = type(odd.spans[0])(**{**odd.spans[0].__dict__, "length_m": 130e3})
    assert not S.in_envelope(odd)                                   # spans differ
    hot = workloads.surrogate_link(5)
    hot.launch_power_w = [x * 100 for x in hot.launch_power_w]
    assert not S.in_envelope(hot)                                   # +20 dB


def test_drho_feature_is_eq12_scale(S, workloads):
    """Feature 16 is Cr P_tot L_eff B_tot, the exponent of the ISRS tilt of Eq. 12."""
    w = workloads.surrogate_link(11)
    s = w.spans[0]
    alpha = s.alpha_db_km * math.log(10) / 10
    L = s.length_m * 1e-3
    leff = (1 - math.exp(-alpha * L)) / alpha
    f = np.asarray(w.centre_hz)
    btot = (f.max() - f.min()) * 1e-12 * 120 / 119
    want = s.cr_per_w_km_thz * sum(w.launch_power_w) * leff * btot
    assert np.isclose(S.features(w)[0, 16], want)


class _Crash(Exception):
    pass


def test_label_shards_resume_after_a_crash(S, tmp_path):
    """generate_labels writes shard after shard; a run that dies in the third
    shard resumes at it, computes only what is missing and returns the same array."""
    seeds = list(range(100, 110))
    calls = []

    def fake(wls, crash_at=None):
        calls.append(list(wls))
        if crash_at is not None and len(calls) == crash_at:
            raise _Crash()
        return [np.full(4, float(s)) + np.arange(4) for s in wls]

    d = str(tmp_path / "labels")
    with pytest.raises(_Crash):
        S.generate_labels(d, seeds, None, shard_links=3, label_fn=lambda w: fake(w, crash_at=3), make_link=int)
    import json, os
    idx = json.load(open(os.path.join(d, "index.json")))
    assert idx["done"] == [0, 1]
    calls.clear()
    got = S.generate_labels(d, seeds, None, shard_links=3, label_fn=fake, make_link=int)
    assert calls == [[106, 107, 108], [109]]                  # only the missing shards
    assert np.array_equal(got, np.array([np.full(4, float(s)) + np.arange(4) for s in seeds]))
    calls.clear()
    assert np.array_equal(S.generate_labels(d, seeds, None, shard_links=3, label_fn=fake, make_link=int), got)
    assert calls == []                                          # complete: nothing recomputed
    # a shard file that exists but was never entered in the index is recomputed
    idx = json.load(open(os.path.join(d, "index.json")))
    idx["done"].remove(1)
    json.dump(idx, open(os.path.join(d, "index.json"), "w"))
    np.save(os.path.join(d, "shard_00001.npy"), np.zeros((3, 4)))
    assert np.array_equal(S.generate_labels(d, seeds, None, shard_links=3, label_fn=fake, make_link=int), got)
    assert calls == [[103, 104, 105]]
    with pytest.raises(ValueError):                             # files of another run are not mixed in
        S.generate_labels(d, seeds[:-1], None, shard_links=3, label_fn=fake, make_link=int)
