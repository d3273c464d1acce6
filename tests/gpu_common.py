"""Shared set-up for the GPU parity tests: one CUDA-library context and one
oracle context on the same parameters (moduli chosen by each side itself and
checked equal), with keys from the same master seed."""
import numpy as np

import oracle.ckks as O
from paper_2510_03996_gb300 import synth


class Pair:
    def __init__(self, name, rot_steps=()):
        import torch
        from paper_2510_03996_gb300 import fheon as F

        torch.cuda.set_device(0)
        F.use_torch_allocator()
        self.F = F
        self.P = P = synth.params(name)
        self.N = N = 1 << P["logN"]
        self.L = L = len(P["qbits"])
        self.g = F.Context(N, qbits=P["qbits"], pbits=P["pbits"], dnum=P["dnum"], scale=P["scale"],
                           seed=P["seed"], stream=torch.cuda.current_stream().cuda_stream)
        self.o_primes = O.gen_primes(N, P["qbits"] + P["pbits"])
        self.o = O.Ctx(N, self.o_primes[:L], self.o_primes[L:], P["dnum"], P["seed"])
        self.sk, self.pk = self.g.keygen()
        self.s_coeff, self.s_eval = self.o.keygen_sk()
        self.opk = self.o.keygen_pk(self.s_eval)
        self.okeys = {}
        self.add_keys(rot_steps)

    def add_keys(self, steps):
        gs = [self.g.galois_elt(r) for r in steps]
        self.g.galois_keygen(self.sk, gs)
        for g in gs:
            if g not in self.okeys:
                self.okeys[g] = self.o.rotkey(self.s_eval, g)

    def encrypt_both(self, m, nonce, level=None):
        ct = self.g.encrypt(self.pk, self.g.plain_from_coeffs(m, self.L, self.P["scale"]), nonce=nonce)
        oct_ = self.o.encrypt(self.opk, m, nonce)
        if level is not None and level < self.L:
            ct = self.g.drop_level(ct, level)
            oct_ = self.o.drop_level(oct_, level)
        return ct, oct_


def mismatch(a, b):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape, (a.shape, b.shape)
    return int(np.sum(a != b))
