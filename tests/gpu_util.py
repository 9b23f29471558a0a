"""Helpers for the GPU parity tests (device buffers through torch)."""
import numpy as np


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def empty_dev(n, dtype):
    import torch
    return torch.empty(n, dtype=dtype, device="cuda")


def assert_dist_close(got, want, rel, what=""):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    zero = want == 0
    assert np.array_equal(got[zero], want[zero]), f"{what}: oracle 0 must be exactly 0"
    nz = ~zero
    err = np.abs(got[nz] - want[nz]) / want[nz]
    assert (err <= rel).all(), f"{what}: max rel err {err.max() if err.size else 0:.3e} > {rel}"
