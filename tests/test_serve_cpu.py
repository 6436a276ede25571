"""Host-side pieces of the serving loop that need no GPU: arrival process and summary."""
import numpy as np

from paper_1301_7530_gb300 import serve as S


def test_poisson_arrivals_per_client_order_and_rate():
    arr = S.poisson_arrivals(4, 5, rate=100.0, seed=3)
    assert len(arr) == 20 and all(a[0] <= b[0] for a, b in zip(arr, arr[1:]))
    per_client = {}
    for t, c, k in arr:
        per_client.setdefault(c, []).append(k)
    assert all(v == list(range(5)) for v in per_client.values())
    big = S.poisson_arrivals(8, 400, rate=200.0, seed=5)
    last = {}
    for t, c, k in big:
        last[c] = t
    # each client's 400 gaps have mean 8 / 200 s
    assert abs(np.mean(list(last.values())) / 400 - 8 / 200) < 0.004


def test_latency_summary():
    reqs = [S.Request(0, k, arrival=0.1 * k, t_done=0.1 * k + 0.01 * (k + 1), status=0, true_rel_res=1e-9)
            for k in range(10)]
    s = S.latency_summary(reqs)
    assert s["solves"] == 10 and s["failed"] == 0
    assert abs(s["p50_ms"] - 55.0) < 1e-6
    assert abs(s["max_ms"] - 100.0) < 1e-9
