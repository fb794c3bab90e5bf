"""Shared pytest set-up: the ``gpu`` marker and the CUDA-availability gate."""

import pytest


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a)")


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover - torch missing entirely
        return False


def pytest_collection_modifyitems(config, items):
    if _cuda_ok():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
