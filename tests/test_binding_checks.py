"""Argument checks of the Python binding that run before any device work, on
the CPU: the no-allocation selection entry rejects injection tensors of the
wrong type, length or layout, output tensors that are too short, and tensors
that are not on a CUDA device; the device-pointer ln L entry rejects a
hyperpoint tensor that is not a float64 [n, 12] CUDA tensor."""
import numpy as np
import pytest
import torch

import paper_2504_02034_b300 as pkg

TH = np.tile(np.array([70.0, 0.3, 1.0, 1.9, 3.4, 34.0, 3.6, 5.0, 100.0, 2.7, 3.0, 2.0]), (3, 1))


def _inj(n=8, **over):
    d = {k: torch.ones(n, dtype=torch.float64) for k in ("dL", "m1d", "m2d", "log_pi")}
    d.update(over)
    return d


def _call(inj, xi=None, neff=None):
    xi = torch.zeros(3, dtype=torch.float64) if xi is None else xi
    neff = torch.zeros(3, dtype=torch.float64) if neff is None else neff
    pkg.chimera_selection_static(TH, inj, 100, 0.039, 1.1, 1.5, xi, neff)


@pytest.mark.parametrize("name", ["m1d", "m2d", "log_pi"])
def test_float32_injection_tensor_rejected(name):
    with pytest.raises(ValueError, match=name):
        _call(_inj(**{name: torch.ones(8, dtype=torch.float32)}))


@pytest.mark.parametrize("name", ["m1d", "m2d", "log_pi"])
def test_short_injection_tensor_rejected(name):
    with pytest.raises(ValueError, match="8 elements"):
        _call(_inj(**{name: torch.ones(7, dtype=torch.float64)}))


def test_non_contiguous_injection_tensor_rejected():
    with pytest.raises(ValueError, match="contiguous"):
        _call(_inj(dL=torch.ones(16, dtype=torch.float64)[::2]))


@pytest.mark.parametrize("which", ["xi", "neff"])
def test_short_output_rejected(which):
    short = torch.zeros(2, dtype=torch.float64)
    with pytest.raises(ValueError, match=">= 3 elements"):
        _call(_inj(), **{which: short})


def test_host_tensors_rejected():
    with pytest.raises(ValueError, match="CUDA"):
        _call(_inj())


def test_device_entry_rejects_host_or_misshaped_theta():
    out = torch.zeros(3, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensor of shape"):
        pkg.chimera_loglike_device(None, 0, torch.zeros(3, 12, dtype=torch.float64), pkg.MIXED, out)
    with pytest.raises(ValueError, match="CUDA tensor of shape"):
        pkg.chimera_loglike_device(None, 0, torch.zeros(3, 11, dtype=torch.float64), pkg.MIXED, out)
    with pytest.raises(ValueError, match="CUDA tensor of shape"):
        pkg.chimera_loglike_device(None, 0, torch.zeros(3, 12, dtype=torch.float32), pkg.MIXED, out)
