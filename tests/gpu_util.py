"""Helpers shared by the GPU tests: device copies and seeded PIR instances."""
import numpy as np

import synth


def to_dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a.reshape(-1)).cuda()


def empty_u32(count):
    import torch
    return torch.empty(int(count), dtype=torch.int32, device="cuda")


def from_dev(t, shape=None):
    import torch
    torch.cuda.synchronize()
    a = t.cpu().numpy().view(np.uint32)
    return a.reshape(shape) if shape is not None else a


def random_queries(P, B, seed):
    """Uniform ciphertext residues [B][D1][2][L][n] (the scan is data independent)."""
    return synth.uniform_residues(seed, synth.STREAM_UNIFORM, B * P.D1 * 2, P.n, P.qs).reshape(B, P.D1, 2, P.L, P.n)


def encrypted_queries(O, P, B, seed):
    """B real one-hot queries; returns (queries, secret, [(i*, c*)])."""
    idx = synth.query_indices(seed, B, P.D1, P.D2)
    s = synth.ternary_secret(seed, P.n)
    out = np.empty((B, P.D1, 2, P.L, P.n), dtype=np.uint32)
    targets = []
    for b in range(B):
        a = synth.uniform_residues(seed, synth.STREAM_A, P.D1, P.n, P.qs, start=b * P.D1)
        e = synth.gaussian_error(seed, P.D1 * P.n, start=b * P.D1 * P.n).reshape(P.D1, P.n)
        i_star, c_star = divmod(int(idx[b]), P.D2)
        out[b] = O.encrypt_query(P, s, a, e, i_star)
        targets.append((i_star, c_star))
    return out, s, targets
