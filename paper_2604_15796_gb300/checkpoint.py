"""Checkpoint and resume of a reconstruction (Algorithm 1): the ADMM state
after iteration k (the contrast m and the TV variables g, u, on the
inversion mesh) and the iteration's weights, saved to a ``.npz`` file that a
later process resumes from.

Every iteration solves its fields from zero at the current contrast, and
the library's results do not depend on the tile variants or the chaining it
picks, so a resumed run repeats the uninterrupted one bit for bit."""
import json

import numpy as np


def save(path, k, m, g, u, params=None):
    """Write the state after iteration ``k``; m, g, u are device tensors."""
    np.savez(path, k=np.int64(k), m=m.detach().cpu().numpy(), g=g.detach().cpu().numpy(),
             u=u.detach().cpu().numpy(), params=np.array(json.dumps(params or {})))


def load(path, device="cuda"):
    """(k, m, g, u, params) of a checkpoint, the tensors on ``device``."""
    import torch
    with np.load(path) as z:
        k = int(z["k"])
        m, g, u = (torch.from_numpy(np.ascontiguousarray(z[n])).to(device) for n in "mgu")
        params = json.loads(str(z["params"]))
    return k, m, g, u, params
