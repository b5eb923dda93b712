"""Helpers for the GPU parity tests: build/load the library, run the oracle, compare.

Error measure (the relative H error of the metric): e_inf = max_i |H_i - H_i^ref|_2 /
max_i |H_i^ref|_2 over cells i, vectors in R^3. The FP32 path must reach <= 1e-5
against the FP64 oracle on the same FP32-rounded input.
"""
import numpy as np

TOL_FP32 = 1e-5


def lib():
    from paper_2308_08447_gb300 import build, gbdemag
    build.build()
    gbdemag.load()
    return gbdemag


def e_inf(H, Href):
    H = np.asarray(H, np.float64)
    Href = np.asarray(Href, np.float64)
    num = np.sqrt(((H - Href) ** 2).sum(axis=0)).max()
    den = np.sqrt((Href ** 2).sum(axis=0)).max()
    return num / den


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)
