"""Writes oracle_tiny_digests.json: SHA-256 digests of the oracle's integer
outputs on the `tiny` parameter set (keys, an encryption, a rotation, a key
switch, a product with relinearisation, a rescale) for fixed seeds.  Calls
only the oracle and the seeded input generators; run it only when a change
to the oracle's arithmetic is justified by the paper or a reading of it,
and name that passage in the commit.

    python tests/golden/make_oracle_digests.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import ckks  # noqa: E402
from paper_2510_03996_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny_digests.json")


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


def compute():
    P = synth.params("tiny")
    N = 1 << P["logN"]
    L = len(P["qbits"])
    mods = ckks.gen_primes(N, P["qbits"] + P["pbits"])
    ctx = ckks.Ctx(N, mods[:L], mods[L:], P["dnum"], P["seed"])
    s, se = ctx.keygen_sk()
    pk = ctx.keygen_pk(se)
    g = ckks.galois_elt(3, N)
    rk = ctx.rotkey(se, g)
    rlk = ctx.relinkey(se)
    m1 = synth.small_int_poly(0x901D, 0, N, 1 << 30)
    m2 = synth.small_int_poly(0x901D, 1, N, 1 << 30)
    c1, c2 = ctx.encrypt(pk, m1, 1), ctx.encrypt(pk, m2, 2)
    return {
        "moduli": digest(np.array(mods, dtype=np.uint64)),
        "secret_key": digest(se),
        "public_key": digest(pk),
        "rotation_key_step_3": digest(rk),
        "relinearisation_key": digest(rlk),
        "encryption": digest(c1),
        "rotation_step_3_level_4": digest(ctx.rotate(c1, g, rk)),
        "rotation_step_3_level_2": digest(ctx.rotate(ctx.drop_level(c1, 2), g, rk)),
        "product_relinearised": digest(ctx.mul_relin(c1, c2, rlk)),
        "rescale": digest(ctx.rescale(c1)),
        "hoisted_steps_1_3": digest(np.stack(ctx.rotate_hoisted(
            c1, [ckks.galois_elt(1, N), g], [ctx.rotkey(se, ckks.galois_elt(1, N)), rk]))),
    }


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(compute(), f, indent=1, sort_keys=True)
        f.write("\n")
    print(OUT)
