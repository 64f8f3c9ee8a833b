"""Shared helpers of the tests: problems built from the seeded draws by the
oracle's twin experiment (inputs never come from the CUDA path)."""
import os

import numpy as np

import eda_synth as S
import oracle as O


def problem(spec, seed=None):
    """(taps, xb, y) of ``spec`` from the oracle's identical twin."""
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    dr = S.draws(spec, seed)
    _, xb, y = O.twin(spec, dr, taps)
    return taps, xb, y


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rowrel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-300)


class env:
    """Temporarily set environment variables (the library reads its tiling
    overrides when a handle is created)."""

    def __init__(self, **kw):
        self.kw = {k: str(v) for k, v in kw.items()}
        self.old = {}

    def __enter__(self):
        for k, v in self.kw.items():
            self.old[k] = os.environ.get(k)
            os.environ[k] = v
        return self

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
