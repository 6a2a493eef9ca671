"""CPU: the serving loop's admission rule (latency-aware, first-in first-out prediction) on
synthetic arrival streams, against a simulated first-in first-out server of known rate."""
import numpy as np

from paper_2301_11376_gb300.serve import LatencyAdmission


def _simulate(rate_true, rate_pred, budget_s, arrivals, samples, alpha=0.0):
    """One server, first in first out, serving `samples[k]` at `rate_true` samples/s.  Requests are
    admitted (or shed) at their arrival time by LatencyAdmission.  Returns latencies of the admitted
    requests, the number shed, the final rate estimate and the admitted samples."""
    adm = LatencyAdmission(budget_s, rate_pred, alpha=alpha, max_in_system=None)
    queue = []          # (completion time, samples) of admitted requests, in order
    busy_until = 0.0
    lat, shed, work = [], 0, 0
    for t, s in zip(arrivals, samples):
        # completions up to now leave the backlog, and report their service
        while queue and queue[0][0] <= t:
            done_t, ds, start = queue.pop(0)
            adm.observe(ds, done_t - start)
            adm.done(ds)
        if not adm.admit(t, t, s):
            shed += 1
            continue
        start = max(t, busy_until)
        busy_until = start + s / rate_true
        queue.append((busy_until, s, start))
        lat.append(busy_until - t)
        work += s
    return np.asarray(lat), shed, adm.rate, work


def _stream(seed, n, mean_gap, mean_samples):
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(mean_gap, n))
    samples = rng.integers(int(0.2 * mean_samples), int(1.8 * mean_samples), n)
    return arrivals, samples


def test_admitted_requests_meet_the_budget_under_overload():
    """Offered load 2.4x capacity: with an exact rate every admitted request finishes within the
    budget (the backlog counts unfinished work in full, so the prediction never undershoots), and
    the server still runs near capacity."""
    rate = 4.5e11
    arrivals, samples = _stream(1, 4000, 0.5e-3, 5.4e8)  # ~1080 Gsamples/s offered
    lat, shed, _, work = _simulate(rate, rate, 0.05, arrivals, samples)
    assert samples.sum() / arrivals[-1] > 2 * rate  # offered load
    assert lat.max() <= 0.05 + 1e-12
    assert 0.4 * len(samples) < shed < 0.75 * len(samples)
    # busy nearly all the time: the admitted work fills most of the run at the server's rate
    assert work / rate > 0.9 * arrivals[-1]


def test_no_shedding_below_capacity():
    rate = 4.5e11
    arrivals, samples = _stream(2, 600, 1.0 / 300, 5.4e8)  # ~160 Gsamples/s offered
    lat, shed, _, _ = _simulate(rate, rate, 0.05, arrivals, samples)
    assert shed == 0 and lat.max() < 0.02


def test_a_flat_bound_sheds_beyond_it_and_keeps_latency_unbounded():
    """Without a budget only the bound on requests in the system sheds; under overload latency then
    grows to the bound over the rate (Little's law), far past any per-frame budget."""
    adm = LatencyAdmission(None, 4.5e11, max_in_system=3)
    assert [adm.admit(0.0, 0.0, 10) for _ in range(5)] == [True, True, True, False, False]
    adm.done(10)
    assert adm.admit(0.0, 0.0, 10) and adm.backlog == 30 and adm.in_system == 3


def test_optimistic_rate_is_corrected_by_observed_service():
    """A calibration 2x too optimistic admits too much at first; observing completed service moves the
    estimate to the true rate, after which admitted requests meet the budget again."""
    rate = 4.5e11
    arrivals, samples = _stream(3, 6000, 0.5e-3, 5.4e8)
    lat, shed, est, _ = _simulate(rate, 2 * rate, 0.05, arrivals, samples, alpha=0.2)
    assert abs(est / rate - 1.0) < 1e-6
    tail = lat[len(lat) // 2:]
    assert tail.max() <= 0.05 + 1e-12


def test_prediction_waits_count():
    """Time already spent waiting counts against the budget."""
    adm = LatencyAdmission(0.010, 1e9, max_in_system=None)
    assert adm.predicted_latency(0.004, 0.0, 5e6) == 0.004 + 5e6 / 1e9
    assert adm.admit(0.0, 0.0, 9e6)            # 9 ms
    assert not adm.admit(0.0005, 0.0, 1e6)     # 0.5 + 9 + 1 ms > 10 ms
    assert adm.admit(0.0, 0.0, 1e6)            # exactly 10 ms
