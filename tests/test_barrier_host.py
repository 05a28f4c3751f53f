"""Host check of the grid barrier's arrival arithmetic (no GPU): block 0 adds
2^31 - (G - 1) to a 32-bit counter and every other block adds 1.  In any arrival
order, bit 31 must stay as it was until the last of the G blocks has arrived, then
differ from the value every block's own add returned, and the low 31 bits must come
back to where they started, so consecutive barriers and launches need no reset."""
import numpy as np

MASK = 0xFFFFFFFF
TOP = 0x80000000


def _add(G, b):
    return (TOP - (G - 1)) & MASK if b == 0 else 1


def test_flip_exactly_at_the_last_arrival_in_any_order():
    rng = np.random.default_rng(0)
    for G in (1, 2, 3, 152, 304, 1024, 4096):
        counter = 0
        for barrier in range(6):
            start = counter
            order = rng.permutation(G)
            olds = []
            for k, b in enumerate(order):
                olds.append(counter)
                # every block that arrives before the last one sees the starting bit 31
                assert ((counter ^ start) & TOP) == 0, (G, barrier, k)
                counter = (counter + _add(G, int(b))) & MASK
                if k < G - 1:
                    # nobody may pass yet
                    assert ((counter ^ start) & TOP) == 0, (G, barrier, k)
            # all arrived: every block sees the flip
            assert all(((o ^ counter) & TOP) != 0 for o in olds), (G, barrier)
            assert (counter & ~TOP & MASK) == (start & ~TOP & MASK)
            assert ((counter ^ start) & TOP) != 0


def test_a_missing_block_never_releases_the_others():
    G = 304
    counter = 0
    olds = []
    for b in range(1, G):          # block 0 never arrives
        olds.append(counter)
        counter = (counter + _add(G, b)) & MASK
    assert all(((o ^ counter) & TOP) == 0 for o in olds)
    counter, olds = 0, []
    for b in range(G - 1):         # the last block never arrives
        olds.append(counter)
        counter = (counter + _add(G, b)) & MASK
    assert all(((o ^ counter) & TOP) == 0 for o in olds)
