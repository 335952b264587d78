"""Host-side check of the schedule the column-block pipelined tree uses
(Sec. 3.1, the reduce loop of Alg. 1; csrc/tree_pipe.cu): merges numbered
level by level, each merge's producers (the last merges into its two slots)
found by the same rule as the kernel, and every wait pointing at a merge with
a lower number -- the property that, with all thread blocks resident, lets
the lowest unfinished merge always proceed.  The slot bookkeeping below is a
plain replay of the tree (the left slot keeps the merged R), independent of
the rule under test."""
import pytest


def merges_at(P, step):
    return (P - step + 2 * step - 1) // (2 * step)


def schedule(P):
    order = []
    step = 1
    while step < P:
        for j in range(merges_at(P, step)):
            left = 2 * j * step
            order.append((step, left, left + step))
        step *= 2
    return order


def producers(P, step, left, right):
    """The kernel's rule: top child = merge (step / 2, left), i.e. counter
    left + step / 2; bottom = the last merge whose left slot is `right`."""
    top = left + step // 2 if step > 1 else None
    bot = None
    st = step // 2
    while st >= 1:
        if right % (2 * st) == 0 and right + st < P:
            bot = right + st
            break
        st //= 2
    return top, bot


@pytest.mark.parametrize("P", list(range(2, 70)) + [127, 128, 129, 152, 255, 256, 300, 304, 513, 1216, 2047])
def test_producers_are_the_last_writers_and_come_first(P):
    order = schedule(P)
    number = {right: i for i, (_, _, right) in enumerate(order)}   # merges are named by their right slot
    assert len(number) == len(order) == P - 1
    last_writer = {}                                                # slot -> merge that last merged into it
    for i, (step, left, right) in enumerate(order):
        assert right < P
        top, bot = producers(P, step, left, right)
        expect_top = order[last_writer[left]][2] if left in last_writer else None
        expect_bot = order[last_writer[right]][2] if right in last_writer else None
        assert (top, bot) == (expect_top, expect_bot)
        for pr in (top, bot):
            if pr is not None:
                assert number[pr] < i                               # waits only on lower numbers
        last_writer[left] = i
    assert order[-1][1] == 0                                        # the root merge ends in slot 0


@pytest.mark.parametrize("P,G", [(304, 304), (152, 302), (1216, 304), (65, 64)])
def test_units_of_a_merge_run_in_the_same_round(P, G):
    """Two thread blocks per merge (units 2m, 2m + 1) and a grid stride G that
    is a multiple of 2: both units of a merge are taken in the same round."""
    K = 2
    G -= G % K
    units = (P - 1) * K
    for u in range(0, units, K):
        assert u // G == (u + K - 1) // G
