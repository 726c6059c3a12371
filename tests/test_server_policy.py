"""The serving loop's scheduling policy, replayed on the host through the C ABI
(eot_server_simulate shares the server's pick function): no GPU needed."""
import numpy as np
import pytest

GB = 1 << 30


@pytest.fixture(scope="module")
def eot():
    from paper_2506_14780_gb300 import eot as e
    e.load()
    return e


def _stream_with_one_large(rate=50.0, duration=20.0, t_large=0.5, seed=0):
    """Small requests (1 GB, 0.2 s each) arriving as a Poisson stream at a
    rate that keeps every slot busy, and one large request (6 GB, 1 s)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, int(rate * duration)))
    n = t.shape[0]
    arrive = np.concatenate([t, [t_large]])
    fp = np.concatenate([np.full(n, GB), [6 * GB]])
    work = np.concatenate([np.full(n, 1.0), [100.0]])
    serv = np.concatenate([np.full(n, 0.2), [1.0]])
    return arrive, fp, work, serv


def test_large_request_is_not_starved(eot):
    """With 8 GB and 8 slots, small 1 GB requests always fit and have less
    predicted work, so shortest-job-first alone would pass the 6 GB request
    over for as long as the stream lasts; once it has waited 1 s the server
    stops admitting others until memory for it has freed up."""
    arrive, fp, work, serv = _stream_with_one_large()
    st, t0, t1 = eot.eot_server_simulate(arrive, fp, work, serv, 8 * GB, 8, max_wait_s=1.0)
    assert st == 0
    wait_large = t0[-1] - arrive[-1]
    # it goes once 1 s has passed and the running small solves (<= 0.2 s) end
    assert 1.0 <= wait_large <= 1.0 + 0.2 + 1e-6, wait_large
    # without the age rule (a wait limit longer than the stream) it waits
    # until the stream of small requests stops
    st, u0, _ = eot.eot_server_simulate(arrive, fp, work, serv, 8 * GB, 8, max_wait_s=1e9)
    assert u0[-1] - arrive[-1] > 15.0
    # every request ran, none overlapping the memory budget
    assert np.all(t0 >= arrive) and np.all(t1 >= t0)


def test_budget_and_slots_are_respected(eot):
    rng = np.random.default_rng(1)
    k = 300
    arrive = np.sort(rng.uniform(0, 5, k))
    fp = rng.integers(1, 5, k) * GB
    work = rng.uniform(1, 10, k)
    serv = rng.uniform(0.01, 0.3, k)
    st, t0, t1 = eot.eot_server_simulate(arrive, fp, work, serv, 10 * GB, 4, max_wait_s=0.5)
    assert st == 0
    events = sorted([(x, 1, i) for i, x in enumerate(t0)] + [(x, -1, i) for i, x in enumerate(t1)],
                    key=lambda e: (e[0], e[1]))
    mem = slots = 0
    for _, kind, i in events:
        if kind == 1:
            mem += fp[i]
            slots += 1
            assert mem <= 10 * GB and slots <= 4
        else:
            mem -= fp[i]
            slots -= 1
    assert np.all(t0 >= arrive - 1e-12)


def test_shortest_job_first_and_refusal(eot):
    """Queued requests that fit go in order of predicted work; a request larger
    than the budget is refused (t = -1) without blocking the others."""
    arrive = np.array([0.0, 0.01, 0.02, 0.03, 0.04])
    fp = np.array([GB, GB, GB, 20 * GB, GB])
    work = np.array([5.0, 9.0, 1.0, 1.0, 3.0])
    serv = np.array([1.0, 0.1, 0.1, 0.1, 0.1])
    st, t0, t1 = eot.eot_server_simulate(arrive, fp, work, serv, 4 * GB, 1, max_wait_s=10.0)
    assert st == 0
    assert t0[3] == -1.0 and t1[3] == -1.0
    # request 0 runs first (alone at t = 0); then by work: 2 (1.0), 4 (3.0), 1 (9.0)
    order = np.argsort(t0[[0, 1, 2, 4]])
    assert list(np.array([0, 1, 2, 4])[order]) == [0, 2, 4, 1]
