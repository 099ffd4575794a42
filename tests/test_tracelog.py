"""Tracer log files of sampler traces: names, layout and a lossless round trip."""
import numpy as np
import pytest

from paper_2003_03508_gb300 import tracelog


@pytest.mark.parametrize("K", [2, 4, 16])
def test_theta_names_follow_the_layout(K):
    names = tracelog.theta_names(K)
    assert len(names) == K * K + 6 * K - 1 and len(set(names)) == len(names)
    o = K * (K - 1)
    assert names[0] == "zP_0_1" and names[o - 1] == f"zP_{K - 1}_{K - 2}"
    assert names[o] == "zpi_1" and names[o + K - 1] == "logit_p_0"
    assert names[o + (K - 1) + K] == "mu_x_0" and names[o + (K - 1) + K + 1] == "mu_y_0"
    assert names[-1] == f"atanh_rho_{K - 1}"


def test_roundtrip(tmp_path):
    rng = np.random.default_rng(0)
    K, C, n = 3, 4, 25
    D = K * K + 6 * K - 1
    lp = rng.normal(-1e4, 30, (n, C))
    th = rng.normal(0, 1, (n, C, D)).astype(np.float32)
    p = tracelog.write_tracer_log(tmp_path / "c2.log", lp, th, K=K, chain=2, first_state=1000, every=10,
                                  comment="K=3 test\nsecond line")
    text = p.read_text().splitlines()
    assert text[0] == "# K=3 test" and text[1] == "# second line"
    assert text[2].split("\t")[:3] == ["state", "posterior", "zP_0_1"]
    cols, states, vals = tracelog.read_tracer_log(p)
    assert cols == ["posterior"] + tracelog.theta_names(K)
    assert list(states) == list(range(1000, 1000 + 10 * n, 10))
    assert np.array_equal(vals[:, 0], lp[:, 2])
    assert np.array_equal(vals[:, 1:], th[:, 2, :].astype(np.float64))


def test_logpost_only_and_errors(tmp_path):
    lp = np.arange(5.0)
    cols, states, vals = tracelog.read_tracer_log(tracelog.write_tracer_log(tmp_path / "a.log", lp))
    assert cols == ["posterior"] and list(states) == [0, 1, 2, 3, 4] and np.array_equal(vals[:, 0], lp)
    with pytest.raises(ValueError):
        tracelog.write_tracer_log(tmp_path / "b.log", lp, np.zeros((5, 7)))          # K missing
    with pytest.raises(ValueError):
        tracelog.write_tracer_log(tmp_path / "b.log", lp, np.zeros((5, 7)), K=2)     # 7 != 15 columns
    with pytest.raises(ValueError):
        tracelog.write_tracer_log(tmp_path / "b.log", lp, np.zeros((4, 15)), K=2)    # n_iter mismatch
