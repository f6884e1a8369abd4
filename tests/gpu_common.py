"""Shared set-up of the GPU parity tests: seeded pencils, gaps from the oracle, and
conversions between numpy blocks and CUDA tensors."""
import numpy as np
import pytest

from oracle import eigs as E
import synth

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.complex128)).cuda()


def host(T):
    torch.cuda.synchronize()
    return T.cpu().numpy()


def colrel(Y, R):
    """max over columns of ||Y_c - R_c|| / ||R_c||."""
    return float(np.max(np.linalg.norm(Y - R, axis=0) / np.maximum(np.linalg.norm(R, axis=0), 1e-300)))


CASES = {
    # name: (builder, leaf_max, eigen-index window for the gaps)
    "real2d_12": (lambda: synth.pencil_2d_real(12, seed=1), 8, (20, 36)),
    "real2d_40": (lambda: synth.pencil_2d_real(40, seed=1), 32, (100, 120)),
    "cplx3d_9": (lambda: synth.pencil_3d_peierls(9, seed=2, wells=6), 16, (40, 70)),
    "cplx3d_12": (lambda: synth.pencil_3d_peierls(12, seed=2, wells=8), 32, (100, 140)),
}


def case(name):
    build, leaf, (p, q) = CASES[name]
    pen = build()
    lam, _ = E.dense_eigs(pen.A, pen.B)
    gaps = (lam[p - 1], lam[p], lam[q - 1], lam[q])
    return pen, leaf, gaps, lam
