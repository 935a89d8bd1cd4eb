"""Shared helpers of the GPU parity tests (inputs and oracle objects only)."""
import numpy as np

from oracle.oracle import Oracle, project_parity
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I


def make(dims, seed=3, eps=0.4, antip=True, recon=18, mass=None):
    fat, lng = I.hisq_links(dims, seed, eps)
    o = Oracle(dims, fat, lng, t_antiperiodic=antip)
    ctx = H.hisq_create(dims, t_antiperiodic=antip, device=0)
    H.hisq_load_links(ctx, fat, lng, long_recon=recon, long_scale=I.C3_NAIK if recon != 18 else 1.0)
    if mass is not None:
        H.hisq_set_mass(ctx, mass)
    return ctx, o


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def dslash_ref(o, dims, field, out_parity):
    return project_parity(dims, o.dslash(project_parity(dims, field, 1 - out_parity)), out_parity)
