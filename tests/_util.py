"""Shared helpers of the GPU tests: seeded inputs and host/device transfers."""
import json
import os

import numpy as np

import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def to_host(t):
    return t.detach().cpu().numpy()


def rel_err(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def mcrit_table():
    path = os.path.join(GOLDEN, "mcrit.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def thermal_links(L, beta=6.0, sweeps=2000, workload_id=0):
    U, theta, acc = inputs.schwinger_links(L, beta, sweeps=sweeps, workload_id=workload_id)
    return U, theta


def mcrit_for(L, beta, workload_id, U=None, theta=None):
    """m_c of a generated field from the stored table (checked by the field digest), else None."""
    key = f"w{workload_id}_L{L}_b{beta:g}"
    row = mcrit_table().get(key)
    if row is None:
        return None
    if theta is not None and row["theta_digest"] != inputs.field_digest(theta):
        return None
    return row["m_crit"]
