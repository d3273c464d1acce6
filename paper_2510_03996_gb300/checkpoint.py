"""Key and ciphertext checkpoints: raw canonical limbs behind a small header.

FHEON keeps its evaluation keys in storage and loads (then clears) the keys
of each network block as it runs (paper Sec. 5.7).  This module is that
storage for the library's keys and ciphertexts.  A file is

    8 bytes   magic b"FHEONCK1"
    8 bytes   little-endian u64: length H of the header
    H bytes   UTF-8 JSON header (kind, N, moduli, and the per-kind fields)
    payload   little-endian u64 limbs, starting on an 8-byte boundary

kind "keys": entries of u64[beta][2][L+K][N] (the layout of
``fheon_key_download``), one per Galois element in the header's
``galois`` list, in that order.  kind "ciphertext": one u64[2][level][N].
A file loads only into a context with the same ring dimension and moduli
(and the same digit split, for keys); residues are checked against their
moduli on the way in.  Keys stream one at a time (memory-mapped), so a
key set far larger than host memory saves and loads.
"""
import json
import os

import numpy as np

MAGIC = b"FHEONCK1"
VERSION = 1


class CheckpointError(ValueError):
    pass


# ---------------------------------------------------------------- file format
def _pad(n):
    return (-n) % 8


def write_header(f, meta):
    """Write magic, length and JSON header; return the payload offset."""
    meta = dict(meta, version=VERSION)
    h = json.dumps(meta, sort_keys=True).encode()
    h += b" " * _pad(len(MAGIC) + 8 + len(h))
    f.write(MAGIC)
    f.write(np.uint64(len(h)).astype("<u8").tobytes())
    f.write(h)
    return len(MAGIC) + 8 + len(h)


def read_header(path):
    """(header dict, payload offset) of a checkpoint file."""
    with open(path, "rb") as f:
        if f.read(len(MAGIC)) != MAGIC:
            raise CheckpointError("%s: not a checkpoint (bad magic)" % path)
        raw = f.read(8)
        if len(raw) != 8:
            raise CheckpointError("%s: truncated header" % path)
        n = int(np.frombuffer(raw, dtype="<u8")[0])
        h = f.read(n)
        if len(h) != n:
            raise CheckpointError("%s: truncated header" % path)
    meta = json.loads(h.decode())
    if meta.get("version") != VERSION:
        raise CheckpointError("%s: version %r, expected %d" % (path, meta.get("version"), VERSION))
    return meta, len(MAGIC) + 8 + n


def _write_atomically(path, body):
    """body(f) writes the file through a temporary of its own beside it
    (a unique name, so concurrent saves do not meet), flushed to the disk
    before it replaces `path`, only when body returns; on any error it is
    removed."""
    import tempfile
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), prefix=os.path.basename(path) + ".")
    try:
        with os.fdopen(fd, "wb") as f:
            body(f)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.remove(tmp)
        raise


def key_shape(meta):
    return (meta["beta"], 2, meta["L"] + meta["K"], meta["N"])


def _expect_size(path, off, count):
    want = off + 8 * count
    got = os.path.getsize(path)
    if got != want:
        raise CheckpointError("%s: %d bytes, the header describes %d" % (path, got, want))


def check_residues(limbs, moduli, axis_limb):
    """Every residue below its limb's modulus (limb index along `axis_limb`)."""
    q = np.asarray(moduli, dtype=np.uint64)
    shape = [1] * limbs.ndim
    shape[axis_limb] = len(q)
    if limbs.shape[axis_limb] != len(q) or not np.all(limbs < q.reshape(shape)):
        raise CheckpointError("a residue is not below its modulus")


def write_keys(path, meta, items):
    """Stream (galois, u64[beta][2][L+K][N]) pairs into a "keys" file.
    `meta` holds N, L, K, alpha, beta, dnum and moduli; `items` may be a
    generator, and its Galois elements are listed in `meta["galois"]`."""
    meta = dict(meta, kind="keys")
    shape = key_shape(meta)

    def body(f):
        write_header(f, meta)
        seen = []
        for g, a in items:
            a = np.ascontiguousarray(a, dtype="<u8")
            if a.shape != shape:
                raise CheckpointError("key %d has shape %s, not %s" % (g, a.shape, shape))
            f.write(a.tobytes())
            seen.append(int(g))
        if seen != [int(g) for g in meta["galois"]]:
            raise CheckpointError("keys written %s differ from the header's list %s" % (seen, meta["galois"]))
    _write_atomically(path, body)


def iter_keys(path, moduli=None):
    """Yield (galois, memory-mapped u64[beta][2][L+K][N]) from a "keys" file,
    checking each key's residues against the file's moduli (or `moduli`)."""
    meta, off = read_header(path)
    if meta.get("kind") != "keys":
        raise CheckpointError("%s holds %r, not keys" % (path, meta.get("kind")))
    shape = key_shape(meta)
    per = int(np.prod(shape))
    _expect_size(path, off, per * len(meta["galois"]))
    mods = list(moduli if moduli is not None else meta["moduli"])
    for i, g in enumerate(meta["galois"]):
        a = np.memmap(path, dtype="<u8", mode="r", offset=off + 8 * per * i, shape=shape)
        check_residues(a, mods, 2)
        yield int(g), a


def write_ct(path, meta, limbs):
    """A "ciphertext" file: u64[2][level][N] with N, level, scale and the
    moduli of its level."""
    a = np.ascontiguousarray(limbs, dtype="<u8")
    meta = dict(meta, kind="ciphertext")
    if a.shape != (2, meta["level"], meta["N"]):
        raise CheckpointError("ciphertext shape %s, header says (2, %d, %d)" % (a.shape, meta["level"], meta["N"]))

    def body(f):
        write_header(f, meta)
        f.write(a.tobytes())
    _write_atomically(path, body)


def read_ct(path):
    """(header, u64[2][level][N]) of a "ciphertext" file, residues checked."""
    meta, off = read_header(path)
    if meta.get("kind") != "ciphertext":
        raise CheckpointError("%s holds %r, not a ciphertext" % (path, meta.get("kind")))
    shape = (2, meta["level"], meta["N"])
    _expect_size(path, off, int(np.prod(shape)))
    a = np.fromfile(path, dtype="<u8", offset=off).reshape(shape)
    check_residues(a, meta["moduli"][:meta["level"]], 1)
    return meta, a.astype(np.uint64)


# ---------------------------------------------------------------- contexts
def context_meta(ctx):
    """What a file must agree on with the context it loads into."""
    return {"N": ctx.N, "L": ctx.L, "K": ctx.K, "alpha": ctx.alpha, "beta": ctx.beta,
            "moduli": [int(q) for q in ctx.moduli]}


def _match(ctx, meta, fields):
    have = context_meta(ctx)
    bad = [k for k in fields if meta.get(k) != have[k]]
    if bad:
        raise CheckpointError("checkpoint made for another context: %s differ" % ", ".join(bad))


def save_keys(ctx, path, galois=None):
    """Write the context's keys (all resident ones, or the Galois elements
    given; 0 is the relinearisation key), one download at a time."""
    gs = ctx.key_list() if galois is None else [int(g) for g in galois]
    meta = dict(context_meta(ctx), galois=gs)
    write_keys(path, meta, ((g, ctx.key_download(g)) for g in gs))
    return gs


def load_keys(ctx, path, galois=None):
    """Install the file's keys (or those of the Galois elements given) on the
    context; returns the elements loaded."""
    meta, _ = read_header(path)
    _match(ctx, meta, ("N", "L", "K", "alpha", "beta", "moduli"))
    want = None if galois is None else {int(g) for g in galois}
    # all or nothing: every selected key is read and checked before the first
    # is installed
    have = [int(g) for g in meta["galois"]]
    if want is not None and want - set(have):
        raise CheckpointError("%s has no key for %s" % (path, sorted(want - set(have))))
    for g, _ in iter_keys(path, ctx.moduli):
        pass  # iter_keys checks every residue of every key
    done = []
    for g, a in iter_keys(path, ctx.moduli):
        if want is None or g in want:
            ctx.key_upload(g, a)
            done.append(g)
    return done


def save_ct(ctx, ct, path):
    level, scale = ctx.ct_info(ct)
    meta = {"N": ctx.N, "level": level, "scale": scale, "moduli": [int(q) for q in ctx.moduli[:level]]}
    write_ct(path, meta, ctx.ct_download(ct))


def load_ct(ctx, path):
    """A new ciphertext handle on the context holding the file's ciphertext."""
    meta, a = read_ct(path)
    if meta["N"] != ctx.N or meta["level"] > ctx.L or meta["moduli"] != [int(q) for q in ctx.moduli[:meta["level"]]]:
        raise CheckpointError("%s: ciphertext made for another context" % path)
    ct = ctx.ct_create(meta["level"], meta["scale"])
    ctx.ct_upload(ct, a)
    ctx.sync()
    return ct
