"""Shared helpers of the GPU parity tests (input preparation only)."""
import numpy as np
import torch

from paper_1401_6750_gb300 import abi, api, synth

ALL_PRECS = (abi.TSM_F64, abi.TSM_F32, abi.TSM_F16, abi.TSM_BF16)


def gauge(ctx, dims, eps, seed, t_bc=-1, precs=ALL_PRECS, unit=False):
    links = synth.unit_links(dims) if unit else synth.gauge_links(dims, eps, seed)
    return api.Gauge(ctx, links, dims, t_bc, precs), links


def round_to(arr, prec):
    """Round a complex128 array the way the library's pack kernel does
    (double -> float -> storage type, round to nearest even)."""
    if prec == abi.TSM_F64:
        return np.asarray(arr, dtype=np.complex128)
    re = torch.from_numpy(np.ascontiguousarray(np.real(arr))).to(torch.float32)
    im = torch.from_numpy(np.ascontiguousarray(np.imag(arr))).to(torch.float32)
    if prec == abi.TSM_F16:
        re, im = re.to(torch.float16), im.to(torch.float16)
    elif prec == abi.TSM_BF16:
        re, im = re.to(torch.bfloat16), im.to(torch.bfloat16)
    return re.to(torch.float64).numpy() + 1j * im.to(torch.float64).numpy()


def to_device(arr):
    return torch.from_numpy(np.ascontiguousarray(arr)).to("cuda")
