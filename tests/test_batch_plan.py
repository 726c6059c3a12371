"""The host-side schedule of eot_solve_batch (gang sizes, transposed runs),
through the C ABI without a GPU: the planning logic the persistent batch
launch uses, checked against the rules it states."""
import numpy as np
import pytest

MODEL = dict(step_ns=1000.0, fix_ns=5000.0, bar_ns=3000.0)


@pytest.fixture(scope="module")
def eot():
    from paper_2506_14780_gb300 import eot
    eot.load()
    return eot


def _opts(eot):
    return eot.default_options(tol=1e-6, max_iter=200000, eps_start=1e-1)


def test_gangs_are_powers_of_two_within_the_cap(eot):
    rng = np.random.default_rng(0)
    k = 300
    n = np.round(np.exp(rng.uniform(np.log(64), np.log(4096), k))).astype(int)
    m = np.round(np.exp(rng.uniform(np.log(64), np.log(4096), k))).astype(int)
    eps = np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), k))
    for grid, cap in ((304, 32), (64, 8), (8, 1)):
        st, gang, tr = eot.eot_batch_plan(n, m, eps, _opts(eot), grid, **MODEL)
        assert st == eot.EOT_OK
        assert np.all(gang >= 1) and np.all(gang <= cap)
        assert np.all(gang & (gang - 1) == 0)
        assert np.array_equal(tr, (n > m).astype(np.int32))


def test_warm_start_keeps_the_roles(eot):
    n, m, eps = [500, 500, 90], [90, 90, 500], [1e-2] * 3
    st, gang, tr = eot.eot_batch_plan(n, m, eps, _opts(eot), 304, **MODEL, has_f_init=[0, 1, 0])
    assert st == eot.EOT_OK and list(tr) == [1, 0, 0]
    # a g_init without f_init (kind 2) runs transposed whatever the shape: the
    # transposed problem's f is the caller's g
    st, gang, tr = eot.eot_batch_plan(n, m, eps, _opts(eot), 304, **MODEL, has_f_init=[2, 2, 2])
    assert st == eot.EOT_OK and list(tr) == [1, 1, 1]


def test_cost_per_cta_floor(eot):
    """At most 1.25 MB of a problem's cost per CTA unless the gang is capped."""
    sizes = [64, 128, 256, 512, 724, 1024, 1448, 2048, 4096]
    st, gang, _ = eot.eot_batch_plan(sizes, sizes, [1e-1] * len(sizes), _opts(eot), 304, **MODEL)
    assert st == eot.EOT_OK
    for s, G in zip(sizes, gang):
        assert G == 32 or G * 1.25 * 2 ** 20 >= 4.0 * s * s, (s, G)
    assert gang[-1] == 32


def test_larger_problems_never_get_smaller_gangs(eot):
    sizes = np.array([64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096])
    st, gang, _ = eot.eot_batch_plan(sizes, sizes, [3e-3] * len(sizes), _opts(eot), 304, **MODEL)
    assert st == eot.EOT_OK
    assert np.all(np.diff(gang) >= 0), gang


def test_a_lone_large_problem_takes_the_largest_useful_gang(eot):
    """With free barriers and no fixed cost, a single problem is the whole
    makespan: its gang doubles up to the cap."""
    st, gang, _ = eot.eot_batch_plan([2048], [2048], [1e-3], _opts(eot), 304, step_ns=1000.0,
                                     fix_ns=0.0, bar_ns=0.0)
    assert st == eot.EOT_OK and gang[0] == 32
    # a barrier that costs more than the work it splits keeps a small problem on one CTA
    st, gang, _ = eot.eot_batch_plan([64], [64], [1e-1], _opts(eot), 304, step_ns=1000.0,
                                     fix_ns=0.0, bar_ns=1e9)
    assert st == eot.EOT_OK and gang[0] == 1


def test_invalid_plans_are_rejected(eot):
    o = _opts(eot)
    assert eot.eot_batch_plan([0], [5], [1e-2], o, 304, **MODEL)[0] == eot.EOT_EINVAL
    assert eot.eot_batch_plan([5], [5], [-1.0], o, 304, **MODEL)[0] == eot.EOT_EINVAL
    assert eot.eot_batch_plan([5], [5], [1e-2], o, 0, **MODEL)[0] == eot.EOT_EINVAL
    assert eot.eot_batch_plan([5], [5], [1e-2], o, 304, step_ns=0.0, fix_ns=0.0,
                              bar_ns=0.0)[0] == eot.EOT_EINVAL
