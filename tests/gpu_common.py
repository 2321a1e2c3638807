"""Shared helpers of the GPU parity tests: build the library once, convert
workloads into device tensors, compare with the oracle."""
from __future__ import annotations

import functools

import numpy as np

import oracle

TOL_FP64 = 1e-10   # FP64 GPU vs oracle, relative L2
TOL_FP32 = 1e-5    # FP32 cell outputs vs oracle, relative L2
TOL_REFINED = 1e-8  # refined (mixed) solutions vs oracle
TOL_ADJ_ORACLE = 1e-6
TOL_ADJ_FD = 1e-4


@functools.lru_cache(None)
def fem():
    from paper_2212_00964_gb300 import build, fem as F
    build.build()
    return F


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def dev(x, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def oracle_material(kind, E, nu, p=3.0, emin=1e-3):
    return oracle.Material(kind, E, nu, p, emin)
