"""The checkpoint file format on the host: keys and ciphertexts round-trip
bit for bit, the payload is 8-byte aligned, and corrupt, truncated or
foreign files are refused (residue at or above its modulus, bad magic,
short payload, another context's moduli).  The context is a stand-in that
stores keys in a dict, so the save/load logic runs without a GPU."""
import os

import numpy as np
import pytest

from paper_2510_03996_gb300 import checkpoint as CK
from paper_2510_03996_gb300 import synth

MODS = [12289, 40961, 65537, 114689]  # primes = 1 mod 2N for N = 16 (L = 3, K = 1)


class FakeCtx:
    def __init__(self, moduli=MODS, N=16, L=3, K=1, alpha=1, beta=3):
        self.N, self.L, self.K, self.alpha, self.beta = N, L, K, alpha, beta
        self.moduli = list(moduli)
        self.keys = {}
        self.cts = {}

    def key_list(self):
        return sorted(self.keys)

    def key_download(self, g):
        return self.keys[g].copy()

    def key_upload(self, g, a):
        self.keys[g] = np.array(a, dtype=np.uint64)

    def ct_info(self, ct):
        return ct["level"], ct["scale"]

    def ct_download(self, ct):
        return ct["limbs"].copy()

    def ct_create(self, level, scale):
        return {"level": level, "scale": scale, "limbs": None}

    def ct_upload(self, ct, a):
        ct["limbs"] = np.array(a, dtype=np.uint64)

    def sync(self):
        pass


def random_limbs(seed, shape, mods, axis):
    rng = synth.rng(0xC4EC, seed)
    q = np.array(mods, dtype=np.uint64)
    bshape = [1] * len(shape)
    bshape[axis] = len(mods)
    return (rng.integers(0, 2 ** 63, size=shape, dtype=np.uint64) % q.reshape(bshape)).astype(np.uint64)


def test_keys_round_trip_and_alignment(tmp_path):
    ctx = FakeCtx()
    shape = (ctx.beta, 2, ctx.L + ctx.K, ctx.N)
    for i, g in enumerate((0, 5, 25)):
        ctx.keys[g] = random_limbs(i, shape, MODS, 2)
    path = str(tmp_path / "k.ck")
    assert CK.save_keys(ctx, path) == [0, 5, 25]
    meta, off = CK.read_header(path)
    assert off % 8 == 0 and meta["kind"] == "keys" and meta["galois"] == [0, 5, 25]
    other = FakeCtx()
    assert CK.load_keys(other, path) == [0, 5, 25]
    for g in (0, 5, 25):
        assert np.array_equal(other.keys[g], ctx.keys[g])
    # a subset, and a key the file lacks
    third = FakeCtx()
    assert CK.load_keys(third, path, [25]) == [25] and list(third.keys) == [25]
    with pytest.raises(CK.CheckpointError):
        CK.load_keys(FakeCtx(), path, [7])


def test_keys_refused_when_corrupt_truncated_or_foreign(tmp_path):
    ctx = FakeCtx()
    shape = (ctx.beta, 2, ctx.L + ctx.K, ctx.N)
    ctx.keys[5] = random_limbs(3, shape, MODS, 2)
    path = str(tmp_path / "k.ck")
    CK.save_keys(ctx, path)
    raw = bytearray(open(path, "rb").read())
    _, off = CK.read_header(path)
    # residue of limb 2 (block 1) set to its modulus
    bad = bytearray(raw)
    pos = off + 8 * ((1 * (ctx.L + ctx.K) + 2) * ctx.N + 4)
    bad[pos:pos + 8] = int(MODS[2]).to_bytes(8, "little")
    p2 = str(tmp_path / "bad.ck")
    open(p2, "wb").write(bytes(bad))
    with pytest.raises(CK.CheckpointError):
        CK.load_keys(FakeCtx(), p2)
    # truncated payload
    open(p2, "wb").write(bytes(raw[:-8]))
    with pytest.raises(CK.CheckpointError):
        CK.load_keys(FakeCtx(), p2)
    # bad magic
    open(p2, "wb").write(b"X" + bytes(raw[1:]))
    with pytest.raises(CK.CheckpointError):
        CK.read_header(p2)
    # another context's moduli or digit split
    with pytest.raises(CK.CheckpointError):
        CK.load_keys(FakeCtx(moduli=[12289, 40961, 65537, 147457]), path)
    with pytest.raises(CK.CheckpointError):
        CK.load_keys(FakeCtx(alpha=3, beta=1), path)


def test_write_keys_checks_shapes_and_list(tmp_path):
    ctx = FakeCtx()
    meta = dict(CK.context_meta(ctx), galois=[5])
    path = str(tmp_path / "k.ck")
    with pytest.raises(CK.CheckpointError):
        CK.write_keys(path, meta, [(5, np.zeros((1, 2, 4, 16), dtype=np.uint64))])
    with pytest.raises(CK.CheckpointError):
        CK.write_keys(path, meta, [(7, np.zeros((3, 2, 4, 16), dtype=np.uint64))])


def test_ciphertext_round_trip(tmp_path):
    ctx = FakeCtx()
    limbs = random_limbs(9, (2, 2, ctx.N), MODS[:2], 1)
    scale = 2.0 ** 40 * (1 + 2.0 ** -30)
    ct = {"level": 2, "scale": scale, "limbs": limbs}
    path = str(tmp_path / "c.ck")
    CK.save_ct(ctx, ct, path)
    back = CK.load_ct(ctx, path)
    assert back["level"] == 2 and back["scale"] == scale
    assert np.array_equal(back["limbs"], limbs)
    meta, off = CK.read_header(path)
    assert off % 8 == 0 and meta["moduli"] == MODS[:2]
    # another context refuses it; a residue at its modulus is refused
    with pytest.raises(CK.CheckpointError):
        CK.load_ct(FakeCtx(moduli=[40961, 12289, 65537, 114689]), path)
    limbs[1, 1, 0] = MODS[1]
    CK.write_ct(path, {"N": 16, "level": 2, "scale": scale, "moduli": MODS[:2]}, limbs)
    with pytest.raises(CK.CheckpointError):
        CK.read_ct(path)


def test_a_failed_save_leaves_no_file(tmp_path):
    ctx = FakeCtx()
    ctx.keys[5] = random_limbs(4, (ctx.beta, 2, ctx.L + ctx.K, ctx.N), MODS, 2)

    def broken(g):
        raise RuntimeError("download failed")
    ctx.key_download = broken
    path = str(tmp_path / "k.ck")
    with pytest.raises(RuntimeError):
        CK.save_keys(ctx, path)
    assert os.listdir(str(tmp_path)) == []
