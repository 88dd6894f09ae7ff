"""CPU model of the mbarrier protocol of the persistent halo convolution kernel (unet_gemm.cu).

The kernel has five agents: the slab-copy thread, the weight-copy thread, the MMA-issue thread, the
tensor pipe (MMAs complete in issue order, each commit arrives on its barrier) and the epilogue warps.
Barriers complete phases; a wait for completion k uses parity k & 1, which is only valid while the
barrier has completed k or k + 1 phases (a waiter two phases behind would see the wrong parity and
hang until its time limit). The model plays the agents in random interleavings and checks, for the
shapes the network uses (taps per chunk, chunks per tile, weight stages S, slab buffers nbuf, tiles
per CTA L):
  * every parity wait happens while the barrier is at most one phase ahead of it;
  * no weight stage and no slab buffer is overwritten before the MMAs that read it are done;
  * the MMAs of a step find its weights and its chunk's slab landed;
  * every schedule ends (no deadlock).
The copy engine's completions arrive in any order. This checks the protocol, not the kernel's code.
"""
import random

import pytest


def simulate(L, nchunks, taps, S, nbuf, seed, slab_guard=True, weight_guard=True):
    rnd = random.Random(seed)
    nsteps = nchunks * taps
    total = L * nsteps
    nch = L * nchunks
    done = {}

    def c(b):
        return done.get(b, 0)

    def can_wait(b, k):
        assert c(b) <= k + 1, ("parity wrap", b, c(b), k)
        return c(b) >= k + 1

    slab_next = 0       # next chunk whose slab the slab thread copies
    wt_next = 0         # next step whose weights the weight thread copies
    issue_next = 0      # next step the MMA thread issues
    epi_next = 0        # next tile the epilogue drains
    copies = []         # in flight: (barrier, index, chunk or step)
    mmas = []           # in flight, in order: (barrier, index, what)
    landed_slab, landed_wt = set(), set()
    steps_done, chunks_done = 0, 0
    for _ in range(10 ** 6):
        moved = False
        agents = ["slab", "wt", "copy", "issue", "mma", "epi"]
        rnd.shuffle(agents)
        for a in agents:
            if a == "slab" and slab_next < nch:
                gc = slab_next
                # the buffer's last readers are the MMAs of chunk gc - nbuf
                if slab_guard and gc >= nbuf and not can_wait(("sbar", gc % nbuf), (gc - nbuf) // nbuf):
                    continue
                assert gc < nbuf or chunks_done >= gc - nbuf + 1, "slab buffer rewritten early"
                copies.append(("sfull", gc % nbuf, gc))
                slab_next += 1
                moved = True
            elif a == "wt" and wt_next < total:
                gs = wt_next
                st = gs % S
                if weight_guard and gs >= S and not can_wait(("bar", st), gs // S - 1):
                    continue
                assert steps_done >= gs - S + 1, "weight stage rewritten early"
                copies.append(("bfull", st, gs))
                wt_next += 1
                moved = True
            elif a == "copy" and copies:
                b, idx, what = copies.pop(rnd.randrange(len(copies)))
                done[(b, idx)] = c((b, idx)) + 1
                (landed_slab if b == "sfull" else landed_wt).add(what)
                moved = True
            elif a == "issue" and issue_next < total:
                gs = issue_next
                l, i = divmod(gs, nsteps)
                chunk, t = divmod(i, taps)
                gc = l * nchunks + chunk
                st = gs % S
                if i == 0 and l >= 2 and not can_wait(("acce", l & 1), (l >> 1) - 1):
                    continue
                if t == 0 and not can_wait(("sfull", gc % nbuf), gc // nbuf):
                    continue
                if not can_wait(("bfull", st), gs // S):
                    continue
                assert gc in landed_slab and gs in landed_wt, "MMA before its operands landed"
                mmas.append(("bar", st, gs))
                if t == taps - 1:
                    mmas.append(("sbar", gc % nbuf, gc))
                if i == nsteps - 1:
                    mmas.append(("accf", l & 1, l))
                issue_next += 1
                moved = True
            elif a == "mma" and mmas:
                b, idx, what = mmas.pop(0)
                done[(b, idx)] = c((b, idx)) + 1
                if b == "bar":
                    steps_done += 1
                if b == "sbar":
                    chunks_done = what + 1
                moved = True
            elif a == "epi" and epi_next < L:
                if not can_wait(("accf", epi_next & 1), epi_next >> 1):
                    continue
                done[("acce", epi_next & 1)] = c(("acce", epi_next & 1)) + 1
                epi_next += 1
                moved = True
        if (slab_next, wt_next, issue_next, epi_next) == (nch, total, total, L) and not copies and not mmas:
            return
        if not moved:
            raise AssertionError(f"deadlock: slab {slab_next} weights {wt_next} issue {issue_next} epilogue {epi_next}")
    raise AssertionError("no end")


@pytest.mark.parametrize("nchunks,taps", [(1, 1), (1, 5), (1, 9), (2, 9), (3, 9), (6, 9)])
@pytest.mark.parametrize("S,nbuf", [(2, 2), (3, 2), (8, 2), (6, 3), (8, 3)])
def test_halo_pipeline_protocol(nchunks, taps, S, nbuf):
    for L in (1, 2, 3, 5):
        for seed in range(12):
            simulate(L, nchunks, taps, S, nbuf, seed)


@pytest.mark.parametrize("guard", ["slab", "weights"])
def test_model_catches_a_missing_wait(guard):
    """The model is not vacuous: without the slab thread's (or the weight thread's) wait for the
    buffer's last readers, some interleaving rewrites a buffer that MMAs still read."""
    with pytest.raises(AssertionError, match="rewritten early"):
        for seed in range(200):
            simulate(3, 2, 9, 3, 2, seed, slab_guard=guard != "slab", weight_guard=guard != "weights")
