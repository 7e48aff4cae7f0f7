"""Helpers shared by the GPU parity tests (tests only)."""
import numpy as np
import torch

from oracle import squint_sac as o


def split_params(flat, cfg):
    """Flat canonical FP32 vector -> {name: array} in the oracle's parameter order."""
    out = {}
    off = 0
    for name, shape, _, _ in o.param_spec(cfg):
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    assert off == len(flat)
    return out


def post_critic_state(P0, p_gpu, cfg):
    """The oracle's parameters P0 with the GPU's critic group and temperature after an
    update: the state the GPU's actor step read (Alg. 1: the actor step follows the
    critic and temperature steps; the actor group is still P0's)."""
    P = {k: v.copy() for k, v in P0.items()}
    for name, *_ in o.param_spec(cfg):
        if o.group_of(name) in ("critic", "alpha"):
            P[name] = np.array(p_gpu[name], dtype=np.float64)
    return P


def flatten(d, cfg):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, *_ in o.param_spec(cfg)])


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


class LazyRows:
    """Row-indexable view of a device tensor that copies only the rows asked for (oracle input)."""

    def __init__(self, t):
        self.t = t
        self.shape = tuple(t.shape)

    def __getitem__(self, idx):
        ii = torch.as_tensor(np.asarray(idx), device=self.t.device, dtype=torch.long)
        return self.t.index_select(0, ii).cpu().numpy()


def lazy_ring(ring):
    return {k: LazyRows(v) for k, v in ring.items()}


def ring_to_device(ring_cpu):
    return {k: v.cuda() for k, v in ring_cpu.items()}
