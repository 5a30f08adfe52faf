"""Host logic of bench.py: the roofline picks the binding pipe and divides by
its peak; the serving-trace summaries (steady-state rate, slowest
micro-batch, largest admission gap) read the trace columns correctly."""

import numpy as np
import pytest

import bench

KEYS = ("admit_ms", "launch_host_ms", "device_ms", "done_ms", "galaxies", "lane", "backlog_galaxies", "lanes_busy")


def _pk():
    return dict(hbm=6.8e12, hbm_src="measured", sfu=10.0e12, fp32=80.0e12, sm_mhz=2070.0, num_sms=152)


@pytest.mark.parametrize("work,bound,unit", [
    (dict(hbm_bytes=6.8e9, ex2=1.0e9, flops=8.0e9), "hbm", "GB/s"),         # 1 ms of HBM, 0.1 of the others
    (dict(hbm_bytes=6.8e8, ex2=1.0e10, flops=8.0e9), "alu", "Tex2/s"),      # MUFU binds
    (dict(hbm_bytes=6.8e8, ex2=1.0e9, flops=8.0e10), "alu", "TFLOP/s"),     # FP32 binds
])
def test_roofline_picks_the_binding_pipe(work, bound, unit):
    r = bench.roofline(work, 2.0, _pk(), "k")
    assert r["bound"] == bound and r["unit"] == unit
    assert r["frac"] == pytest.approx(0.5)          # each case has 1 ms of work on its pipe, timed at 2 ms
    assert max(r["fractions"].values()) == pytest.approx(0.5)
    assert r["achieved"] == pytest.approx(r["frac"] * r["peak"])


def _trace(done_ms, galaxies, admit_ms=None, device_ms=None):
    n = len(done_ms)
    tr = np.zeros((n, len(KEYS)))
    tr[:, 0] = admit_ms if admit_ms is not None else np.asarray(done_ms) - 1.0
    tr[:, 2] = device_ms if device_ms is not None else 0.5
    tr[:, 3] = done_ms
    tr[:, 4] = galaxies
    return tr


def test_steady_rate_leaves_out_start_and_drain():
    # 1000 galaxies per ms in the middle, a slow start and a slow tail
    done = np.concatenate([np.arange(0, 50, 5.0), 50 + np.arange(200) * 1.0, 250 + np.arange(0, 50, 5.0)])
    gal = np.full(len(done), 1000.0)
    gal[:10] = 100.0
    gal[-10:] = 100.0
    rate = bench.trace_steady_rate(_trace(done, gal), KEYS)
    assert rate == pytest.approx(1.0e6, rel=0.02)


def test_steady_rate_order_independent_and_degenerate():
    done = np.arange(100, dtype=float)
    tr = _trace(done, np.full(100, 10.0))
    rng = np.random.default_rng(0)
    assert bench.trace_steady_rate(tr[rng.permutation(100)], KEYS) == pytest.approx(1.0e4, rel=0.02)
    assert bench.trace_steady_rate(tr[:3], KEYS) is None


def test_episode_finds_the_slowest_batch_and_the_largest_gap():
    admit = np.array([0.0, 1.0, 2.0, 12.0, 13.0, 14.0])
    done = admit + np.array([0.5, 0.5, 0.5, 9.0, 0.5, 0.5])
    ep = bench.trace_episode(_trace(done, np.ones(6), admit_ms=admit), KEYS, before=2)
    assert ep["admission_to_done_ms"] == pytest.approx(9.0)
    assert ep["max_admission_gap_ms"] == pytest.approx(10.0)
    assert [row[0] for row in ep["rows"]] == [1.0, 2.0, 12.0]
    assert bench.trace_episode(np.zeros((0, len(KEYS))), KEYS) is None


def test_host_cpu_delta():
    a = {"cpu_s": 1.0, "involuntary_switches": 3, "voluntary_switches": 10}
    b = {"cpu_s": 3.0, "involuntary_switches": 5, "voluntary_switches": 30}
    d = bench.host_cpu_delta(a, b, 4.0)
    assert d["cpu_cores_busy"] == pytest.approx(0.5)
    assert d["involuntary_switches"] == 2 and d["voluntary_switches"] == 20


def test_parse_node_list():
    assert bench.parse_node_list("0\n") == [0]
    assert bench.parse_node_list("0-1,4") == [0, 1, 4]
    assert bench.parse_node_list("") == []
