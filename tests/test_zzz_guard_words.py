"""Guard words around every device block, in place of a memory checker:
the blocks come from a test allocator that pads each one with 4 KiB of a
fixed byte on both sides and never hands memory out twice.  Rotations at
every level, batches at mixed levels and hoisted rotations in every
key-switching schedule, and a product with relinearisation and a rescale
run on it, each output bit-exact against the oracle; then every guard byte
must still hold its value."""
import pytest

import gpu_common
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu

GUARD, BYTE = 4096, 0xA5
STEPS = [1, -1, 7, 100]
SCHEDULES = (0, 1, 2, 3, 4, 5, 6, 7, 9, 11, 13, 15, 17, 25, 31)


class GuardedBlocks:
    """alloc/free hooks over torch tensors; every block stays allocated until
    the test ends, so that all guards can be read at the end."""

    def __init__(self):
        import torch
        self.torch = torch
        self.blocks = []

    def alloc(self, nbytes, stream, user):
        torch, n = self.torch, int(nbytes)
        try:
            t = torch.empty(n + 2 * GUARD, dtype=torch.uint8, device="cuda")
        except Exception:  # out of memory: the library reports FHEON_ERR_OOM
            return None
        t[:GUARD].fill_(BYTE)
        t[GUARD + n:].fill_(BYTE)
        self.blocks.append((t, n))
        return t.data_ptr() + GUARD

    def free(self, ptr, nbytes, stream, user):
        pass

    def damaged(self):
        self.torch.cuda.synchronize()
        return [n for t, n in self.blocks
                if not (bool((t[:GUARD] == BYTE).all()) and bool((t[GUARD + n:] == BYTE).all()))]


def test_guard_words_stay_intact():
    pr = gpu_common.Pair("small_n12")
    g, o, F = pr.g, pr.o, pr.F
    mismatch = gpu_common.mismatch
    guard = GuardedBlocks()
    F.set_allocator(guard.alloc, guard.free)
    try:
        pr.add_keys(STEPS)
        gs = [g.galois_elt(st) for st in STEPS]
        g.relinkeygen(pr.sk)
        orlk = o.relinkey(pr.s_eval)
        for level in range(pr.L, 0, -1):
            m = synth.small_int_poly(31, level, pr.N, 1 << 40)
            ct, oct_ = pr.encrypt_both(m, nonce=4000 + level, level=level)
            for st, ge in zip(STEPS, gs):
                assert mismatch(g.ct_download(g.rotate(ct, st)), o.rotate(oct_, ge, pr.okeys[ge])) == 0

        levels = [5, 3, 1, 4]
        pairs = [pr.encrypt_both(synth.small_int_poly(32, i, pr.N, 1 << 40), nonce=4100 + i, level=lv)
                 for i, lv in enumerate(levels)]
        wants = [o.rotate(oc, ge, pr.okeys[ge]) for (_, oc), ge in zip(pairs, gs)]
        hoisted_wants = o.rotate_hoisted(pairs[0][1], gs, [pr.okeys[ge] for ge in gs])
        old = g.get_schedule()
        try:
            for schedule in SCHEDULES:
                g.set_schedule(schedule)
                outs = [g.ct_create(lv) for lv in levels]
                g.rotate_batch([c for c, _ in pairs], outs, STEPS)
                for out, want in zip(outs, wants):
                    assert mismatch(g.ct_download(out), want) == 0, schedule
                for out, want in zip(g.rotate_hoisted(pairs[0][0], STEPS), hoisted_wants):
                    assert mismatch(g.ct_download(out), want) == 0, schedule
        finally:
            g.set_schedule(old)

        b, ob = pr.encrypt_both(synth.small_int_poly(33, 0, pr.N, 1 << 40), nonce=4200, level=5)
        got = g.rescale(g.mul_relin(pairs[0][0], b))
        assert mismatch(g.ct_download(got), o.rescale(o.mul_relin(pairs[0][1], ob, orlk))) == 0

        g.sync()
        assert len(guard.blocks) > 20
        assert guard.damaged() == []
    finally:
        F.use_torch_allocator()
        g.close()
        guard.blocks.clear()  # the hooks outlive the test; the memory need not
