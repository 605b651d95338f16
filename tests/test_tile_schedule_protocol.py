"""The persistent tile hand-out of the remainder-heavy products, as a host model.

A launch of G CTAs of W warps works on T tiles.  Warp w first takes tile w,
then, after each tile, takes sched[0] (an atomic fetch-and-add) and works on
tile G*W + that value while it is below T.  Each CTA, once all its warps are
done, adds one to sched[1]; the CTA that sees G - 1 there clears both words.
The model runs the warps in random interleavings (the order in which the GPU
serves the atomics) and checks that every tile is processed exactly once, that
both words are zero after the launch, and that a second launch on the same
words behaves the same -- the properties the kernels rely on, including under
CUDA-graph replay, where no host code runs between launches.
"""
import random

import pytest


def run_launch(G, W, T, sched, rng, first=None):
    done = []
    nw = G * W
    # each warp's state: the tile it works on next (None once finished)
    cur = {(c, k): c * W + k for c in range(G) for k in range(W)}
    for key in cur:
        if cur[key] >= T:
            cur[key] = None
    warps_left = {c: sum(cur[(c, k)] is not None for k in range(W)) for c in range(G)}
    ticketed = set()

    def finish_cta(c):
        t = sched[1]
        sched[1] += 1
        if t == G - 1:
            sched[0] = 0
            sched[1] = 0

    # CTAs whose warps all start beyond T finish at once
    for c in range(G):
        if warps_left[c] == 0:
            ticketed.add(c)
            finish_cta(c)
    active = [k for k, v in cur.items() if v is not None]
    while active:
        key = rng.choice(active)
        if first is not None:
            first.setdefault(key, cur[key])
        done.append(cur[key])         # the warp finishes its tile ...
        t = sched[0]                  # ... and takes a ticket
        sched[0] += 1
        nxt = nw + t
        if nxt < T:
            cur[key] = nxt
        else:
            cur[key] = None
            active.remove(key)
            c = key[0]
            warps_left[c] -= 1
            if warps_left[c] == 0:
                ticketed.add(c)
                finish_cta(c)
    assert ticketed == set(range(G))
    return done


@pytest.mark.parametrize("G,W,T", [(608, 8, 32768), (152, 8, 100), (4, 8, 1), (7, 8, 57),
                                   (608, 8, 4864), (608, 8, 4865), (3, 1, 1000)])
def test_every_tile_once_and_counters_cleared(G, W, T):
    rng = random.Random(G * 1000003 + W * 101 + T)
    sched = [0, 0]
    for launch in range(3):      # back-to-back launches on the same counters
        done = run_launch(G, W, T, sched, rng)
        assert sorted(done) == list(range(T)), launch
        assert sched == [0, 0], launch


def test_static_first_tiles():
    # with at least as many tiles as warps, warp (c, k) starts on tile c W + k:
    # the tile a one-tile-a-warp launch gives it, whatever the interleaving
    rng = random.Random(5)
    G, W, T = 20, 8, 1000
    first = {}
    sched = [0, 0]
    done = run_launch(G, W, T, sched, rng, first)
    assert all(first[(c, k)] == c * W + k for c in range(G) for k in range(W))
    assert sorted(done) == list(range(T)) and sched == [0, 0]
