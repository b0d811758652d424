"""Host scheduler of the batched persistent launch (no GPU): the task list it
hands to the device queue must contain every task of the tiled LU DAG once,
in an order where every dependency comes earlier (the property that lets the
queue progress without co-resident CTAs), with the critical path first."""
import numpy as np
import pytest

from helpers import lib

PANEL, UPDATE, LSWAP, SOLVE = 0, 1, 2, 3


def expected_tasks(nb, m, with_lu, with_solve):
    """Task set of the right-looking tiled LU with partial pivoting, written out
    from its definition: panel k, update of block column j > k by step k,
    interchange fix-up of block column j < nb - 1, solve chunks of 32 columns."""
    out = {}
    for i, (b, mm) in enumerate(zip(nb, m)):
        if with_lu:
            for k in range(b):
                out[(PANEL, i, k, k)] = [(UPDATE, i, k - 1, k)] if k > 0 else []
                for j in range(k + 1, b):
                    out[(UPDATE, i, k, j)] = [(PANEL, i, k, k)] + ([(UPDATE, i, k - 1, j)] if k > 0 else [])
            for j in range(b - 1):
                out[(LSWAP, i, 0, j)] = [(PANEL, i, b - 1, b - 1)]
        if with_solve:
            for c in range((mm + 31) // 32):
                deps = []
                if with_lu:
                    deps = [(PANEL, i, b - 1, b - 1)] + [(LSWAP, i, 0, j) for j in range(b - 1)]
                out[(SOLVE, i, 0, c)] = deps
    return out


@pytest.mark.parametrize("with_lu,with_solve", [(True, False), (True, True), (False, True)])
@pytest.mark.parametrize("seed", [0, 1])
def test_plan_is_a_topological_order_of_the_whole_dag(with_lu, with_solve, seed):
    fg = lib()
    rng = np.random.default_rng(seed)
    nmat = 12
    nb = rng.integers(1, 9, nmat)
    m = rng.integers(1, 130, nmat)
    tasks, makespan = fg.feast_batch_plan(nb, m, with_lu, with_solve, workers=5)
    exp = expected_tasks(nb.tolist(), m.tolist(), with_lu, with_solve)
    got = [tuple(int(v) for v in t) for t in tasks]
    assert len(got) == len(set(got)) == len(exp)
    assert set(got) == set(exp)
    pos = {t: i for i, t in enumerate(got)}
    for t, deps in exp.items():
        for d in deps:
            assert pos[d] < pos[t], (d, t)
    assert makespan > 0


def test_plan_starts_with_the_longest_matrix_and_schedules_within_graham_bound():
    fg = lib()
    nb = [2, 7, 3, 7, 1]
    m = [40, 64, 100, 10, 32]
    W = 4
    tasks, makespan = fg.feast_batch_plan(nb, m, True, True, workers=W)
    # first task: a panel of a matrix with the most block columns (the longest chain)
    assert tasks[0][0] == PANEL and nb[tasks[0][1]] == max(nb)
    # list scheduling: makespan <= total work / W + longest path (Graham)
    def cost(t):
        kind, i, k, j = t
        b = nb[i]
        if kind == PANEL:
            return 8.0 + 0.06 * 64 * (b - k)
        if kind == UPDATE:
            return 3.0 + 4.5 * (b - k - 1)
        if kind == LSWAP:
            return 1.0 + (b - 1 - j)
        w = min(32, m[i] - 32 * j)
        return 6.0 * b + 2.2 * b * (b - 1) * (w / 32.0)
    total = sum(cost(tuple(t)) for t in tasks)
    assert makespan <= total / W + total + 1e-9
    assert makespan >= total / W - 1e-9


def test_solve_only_plan_is_longest_first():
    fg = lib()
    nb = [1, 4, 2, 8, 3]
    m = [32, 32, 32, 32, 32]
    tasks, _ = fg.feast_batch_plan(nb, m, False, True, workers=3)
    order = [nb[t[1]] for t in tasks]
    assert order == sorted(order, reverse=True)


def test_plan_rejects_bad_arguments():
    fg = lib()
    with pytest.raises(fg.FeastError):
        fg.feast_batch_plan([0, 2], [4, 4], True, True, workers=2)
