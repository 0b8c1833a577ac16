"""Host-side checks of the serving loop's plan pool (no GPU: the plans are stand-ins that record
when they are closed).  The pool must admit every request whose plan fits the HBM budget alone, once
the batches ahead of it finish, however the budget was filled by idle plans of other keys."""
import random

import pytest


class FakePlan:
    def __init__(self, key):
        self.key = key
        self.closed = False

    def close(self):
        assert not self.closed
        self.closed = True


@pytest.fixture
def PlanPool():
    from paper_2606_25595_gb300.serve import PlanPool
    return PlanPool


def test_idle_plans_of_other_keys_make_room(PlanPool):
    """Budget 100: two idle 40-byte plans of key A fill 80; a 70-byte plan of key B closes both
    (without the eviction step it would never be admitted)."""
    made = []
    pool = PlanPool(100, lambda k: made.append(FakePlan(k)) or made[-1])
    pool.warm([("A", 40), ("B", 70)], per_key=2)
    assert [p.key for p in made] == ["A", "A"] and pool.used == 80
    p = pool.take("B", 70)
    assert p is not None and p.key == "B"
    assert all(q.closed for q in made[:2]) and pool.used == 70 and pool.evicted == 2


def test_plans_in_use_are_never_closed(PlanPool):
    pool = PlanPool(100, FakePlan)
    a1 = pool.take("A", 40)
    a2 = pool.take("A", 40)
    pool.give(a2)
    assert pool.take("B", 70) is None          # a1 is in use: closing a2 alone leaves 40 + 70 > 100
    assert not a1.closed and a2.closed and pool.used == 40
    pool.give(a1)
    b = pool.take("B", 70)
    assert b is not None and a1.closed and pool.used == 70


def test_same_key_is_reused_before_anything_is_made(PlanPool):
    pool = PlanPool(100, FakePlan)
    a = pool.take("A", 40)
    pool.give(a)
    assert pool.take("A", 40) is a and pool.used == 40


def test_plan_beyond_the_budget_evicts_nothing(PlanPool):
    pool = PlanPool(100, FakePlan)
    a = pool.take("A", 40)
    pool.give(a)
    assert pool.take("B", 101) is None and not a.closed and pool.used == 40


def test_warm_serves_every_key_before_any_key_twice(PlanPool):
    pool = PlanPool(10 + 20 + 30 + 40, FakePlan)
    pool.warm([("a", 10), ("b", 20), ("c", 30), ("d", 40)], per_key=3)
    assert sorted(pool.idle) == ["a", "b", "c", "d"]
    assert all(len(v) == 1 for v in pool.idle.values()) and pool.used == 100


@pytest.mark.parametrize("seed", range(5))
def test_random_request_stream_completes(PlanPool, seed):
    """Requests of random keys on 3 slots, a batch finishing a few polls after it starts: every
    request is admitted within a bounded number of polls and the budget is never exceeded."""
    rng = random.Random(seed)
    need = {"b64": 3, "b128": 7, "b256": 14, "b512": 28}
    budget = 40
    pool = PlanPool(budget, FakePlan)
    pool.warm(list(need.items()), per_key=4)
    queue = [rng.choice(list(need)) for _ in range(200)]
    busy = [None] * 3
    done = polls = 0
    while queue or any(busy):
        polls += 1
        assert polls < 10_000
        for s, item in enumerate(busy):
            if item is not None:
                plans, left = item
                if left == 0:
                    for p in plans:
                        pool.give(p)
                    done += len(plans)
                    busy[s] = None
                else:
                    busy[s] = (plans, left - 1)
        for s in range(len(busy)):
            if busy[s] is not None or not queue:
                continue
            batch = []
            for key in list(queue):
                p = pool.take(key, need[key])
                if p is None:
                    continue
                assert not p.closed
                queue.remove(key)
                batch.append(p)
                if len(batch) == 4:
                    break
            if batch:
                busy[s] = (batch, rng.randrange(3))
        assert pool.used <= budget
    assert done == 200


def test_close_frees_only_idle_plans(PlanPool):
    pool = PlanPool(100, FakePlan)
    a, b = pool.take("A", 30), pool.take("B", 50)
    pool.give(a)
    pool.close()
    assert a.closed and not b.closed and pool.used == 50


def test_key_with_a_plan_in_use_waits_instead_of_evicting(PlanPool):
    pool = PlanPool(100, FakePlan)
    a = pool.take("A", 40)
    b = pool.take("B", 50)
    pool.give(b)
    assert pool.take("A", 40) is None and not b.closed and pool.used == 90
    pool.give(a)
    assert pool.take("A", 40) is a
