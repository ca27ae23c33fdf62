"""Helpers for the GPU parity tests: device copies of numpy arrays."""
import numpy as np


def dev():
    import torch
    return torch.device("cuda:0")


def d64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint64)).view(np.int64)).to(dev())


def d8(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint8))).to(dev())


def h64(t):
    return t.cpu().numpy().view(np.uint64)


def zeros64(*shape):
    import torch
    return torch.zeros(shape, dtype=torch.int64, device=dev())


def zeros8(*shape):
    import torch
    return torch.zeros(shape, dtype=torch.uint8, device=dev())


def rand_nodes(rnd, T, p):
    s = set()
    while len(s) < T:
        s.add(rnd.randrange(1, p))
    return np.array(sorted(s, key=lambda x: rnd.random()), dtype=np.uint64)


def rand_res(rnd, shape, p):
    n = int(np.prod(shape))
    return np.array([rnd.randrange(p) for _ in range(n)], dtype=np.uint64).reshape(shape)
