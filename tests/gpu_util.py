"""Shared helpers of the GPU parity tests: seeded scenes -> device tensors, oracle problems."""
import numpy as np

from oracle import sgp_oracle as O


def dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    elif t.dtype == torch.float64:
        t = t.float()
    return t.cuda()


def host(t):
    return t.detach().double().cpu().numpy()


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_problem(sc, sigma_R=1e-2):
    """FP64 oracle problem built from exactly the arrays the GPU receives (float32-rounded)."""
    psfs = np.asarray(sc.psfs, np.float32).astype(np.float64)
    g = np.asarray(sc.g, np.float32).astype(np.float64)
    return O.Problem(psfs, g, np.asarray(sc.b, np.float32).astype(np.float64), mask_S=sc.mask, sigma_R=sigma_R)


def gpu_problem(lib, sc, params=None):
    p = lib.Problems(dev(np.asarray(sc.psfs, np.float32)), list(np.asarray(sc.b, np.float32)),
                     dev(sc.mask) if sc.mask is not None else None, params)
    p.set_data(0, dev(np.asarray(sc.g, np.float32)))
    return p


def fp32_envelope():
    """Per-iteration bound on the KL deviation of an FP32 SGP run from the FP64 oracle on the
    256^2 star field (tests/golden/sgp_fp32_envelope.json, written from the oracle alone): the
    largest deviation that single-precision transforms cause in the oracle itself, floored at the
    1e-5 operator-level tolerance."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "sgp_fp32_envelope.json")) as fh:
        env = json.load(fh)
    return env, [max(1e-5, x) for x in env["max_rel_J_per_k"]]
