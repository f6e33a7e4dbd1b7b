"""Pins for the oracle's dispatch-protocol simulator and execution-log
checker.  The simulator's correct runs must satisfy every invariant in every
interleaving of tiny instances (exhaustive state-space search); each planted
mistake must be caught; and hand-written logs pin each checker rule.  CPU only."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _golden_table1():
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "table1_mailbox_codes.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                d, name, v = line.split()
                rows.append((d, name, int(v)))
    return rows


def test_table1_codes_in_simulator(oracle_lib):
    from oracle import protocol as P

    for d, name, v in _golden_table1():
        table = P.FROM_GPU if d == "from_GPU" else P.TO_GPU
        assert table[name] == v


def test_table1_codes_in_public_header():
    text = open(os.path.join(ROOT, "include", "lk.h")).read()
    defs = dict(re.findall(r"#define\s+(LK_\w+)\s+(-?\d+)", text))
    names = {"THREAD_INIT": "LK_ST_INIT", "THREAD_FINISHED": "LK_ST_FINISHED", "THREAD_WORKING": "LK_ST_WORKING"}
    for d, name, v in _golden_table1():
        if d == "from_GPU":
            key = names.get(name, "LK_ST_NOP")
        else:
            key = {"THREAD_NOP": "LK_CMD_NOP", "THREAD_EXIT": "LK_CMD_EXIT", "THREAD_WORK": "LK_CMD_WORK"}[name]
        assert int(defs[key]) == v, (name, key)


def _inst(mode, mutate=None, R=2, D=1, sizes=(2, 1), jobs=None):
    from oracle import protocol as P

    smids = tuple(tuple(10 * c + r for r in range(s)) for c, s in enumerate(sizes))
    jobs = jobs or (((0, 1), (1, 2), (0, 3)), ((1, 4), (0, 5)))
    return P.Instance(sizes=sizes, smids=smids, jobs=jobs, mode=mode, ring_depth=R, bcast_depth=D, mutate=mutate)


@pytest.mark.parametrize("mode,R,D", [("ring", 1, 1), ("ring", 2, 1), ("ring", 2, 2), ("mailbox", 1, 1)])
def test_every_interleaving_satisfies_invariants(oracle_lib, mode, R, D):
    from oracle import protocol as P

    terminals, states = P.explore(_inst(mode, R=R, D=D))
    assert states > 100 and len(terminals) >= 2   # producers interleave: several FIFO orders
    for s in terminals:
        res = P.check_state(s)
        assert res["ok"], res
        assert all(s.done[c] == len(s.posted[c]) or mode == "mailbox" for c in range(2))


def test_single_producer_fifo_is_submission_order(oracle_lib):
    from oracle import protocol as P

    jobs = (((0, 1), (0, 2), (0, 3)),)
    terminals, _ = P.explore(_inst("ring", sizes=(2,), jobs=jobs))
    assert len(terminals) == 1
    s = terminals[0]
    for log in s.logs[0]:
        assert [e[1] for e in log] == [1, 2, 3]


RING_MUTATIONS = ["skip_share", "double_share", "wrong_smid", "early_complete", "ignore_bcast_free",
                  "ignore_ring_full", "wrong_op"]


@pytest.mark.parametrize("mutation", RING_MUTATIONS)
def test_planted_mistakes_are_caught_ring(oracle_lib, mutation):
    from oracle import protocol as P

    R = 1 if mutation == "ignore_ring_full" else 2
    terminals, _ = P.explore(_inst("ring", mutate=mutation, R=R))
    caught = [s for s in terminals if not P.check_state(s)["ok"]]
    assert caught, mutation


@pytest.mark.parametrize("mutation", ["skip_share", "double_share", "wrong_smid", "early_complete", "wrong_op"])
def test_planted_mistakes_are_caught_mailbox(oracle_lib, mutation):
    from oracle import protocol as P

    terminals, _ = P.explore(_inst("mailbox", mutate=mutation))
    assert any(not P.check_state(s)["ok"] for s in terminals), mutation


@pytest.mark.parametrize("seed", range(6))
def test_random_interleavings_medium(oracle_lib, seed):
    from oracle import protocol as P

    sizes = (3, 2, 4, 1)
    jobs = tuple(tuple(((p + j) % 4, 1 + (j % 5)) for j in range(12)) for p in range(3))
    inst = P.Instance(sizes=sizes, smids=tuple(tuple(100 + 10 * c + r for r in range(s)) for c, s in enumerate(sizes)),
                      jobs=jobs, mode="ring", ring_depth=4, bcast_depth=2)
    s = P.run_random(inst, seed)
    res = P.check_state(s)
    assert res["ok"], res
    assert sum(len(p) for p in s.posted) == 36


# ---- hand-written logs pin each rule of the checker -------------------------------
def _good_log():
    # 2 clusters: sizes 2 and 1; cluster 0 ran seq 1,2; cluster 1 ran seq 1
    rows = [  # seq cluster rank smid op order
        (1, 0, 0, 5, 1, 0), (2, 0, 0, 5, 2, 1),
        (1, 0, 1, 9, 1, 0), (2, 0, 1, 9, 2, 1),
        (1, 1, 0, 3, 4, 0),
    ]
    return [list(r) for r in rows]


def _check(rows, **kw):
    import oracle

    a = np.array(rows, dtype=np.int64)
    args = dict(cluster_size=[2, 1], n_posted=[2, 1], pinned_smid=[5, 9, 3], posted_op=[1, 2, 4])
    args.update(kw)
    return oracle.check_exec_log(a[:, 0], a[:, 1], a[:, 2], a[:, 3], a[:, 4], a[:, 5], **args)


def test_checker_accepts_good_log(oracle_lib):
    assert _check(_good_log())["violations"] == 0


@pytest.mark.parametrize("edit,code", [
    (lambda r: r.pop(1), "missing"),
    (lambda r: r.append(list(r[0])), "duplicate"),
    (lambda r: (r[0].__setitem__(5, 1), r[1].__setitem__(5, 0)), "fifo"),
    (lambda r: r[2].__setitem__(3, 77), "wrong_sm"),
    (lambda r: r[4].__setitem__(4, 2), "wrong_op"),
    (lambda r: r[4].__setitem__(0, 2), "bad_seq"),
    (lambda r: r[4].__setitem__(1, 5), "bad_cluster"),
    (lambda r: r[4].__setitem__(2, 1), "bad_rank"),
])
def test_checker_flags_each_rule(oracle_lib, edit, code):
    rows = _good_log()
    edit(rows)
    res = _check(rows)
    assert res["violations"] > 0 and code in res["counts"], res


def test_checker_completion_soundness(oracle_lib):
    rows = _good_log()
    t_end = np.array([10, 20, 11, 25, 5], dtype=np.uint64)
    ok = _check(rows, t_end=t_end, t_complete=[12, 26, 6])
    assert ok["violations"] == 0
    bad = _check(rows, t_end=t_end, t_complete=[12, 22, 6])   # seq 2 completed before rank 1 ended
    assert bad["counts"].get("early_complete") == 1
