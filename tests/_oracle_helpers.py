"""Shared set-up for the oracle tests (tiny systems with a brute-force twin)."""
import numpy as np
import torch

from oracle import cc3
from oracle.bruteforce import BruteCC3
from paper_2407_18947_gb300.synth import make_system


def tiny(o, v, seed=7, naux=None):
    s = make_system(o, v, naux=naux, seed=seed)
    ham = cc3.Hamiltonian.from_system(s)
    g = torch.einsum('Ppq,Prs->pqrs', ham.L, ham.L).numpy()
    bf = BruteCC3(s.eps, ham.h.numpy(), g, o)
    return s, ham, bf


def sym_pair(x):
    return 0.5 * (x + x.transpose(1, 0, 3, 2))
