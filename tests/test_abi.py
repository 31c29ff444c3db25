"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/tsbts.h declares. No compute call needs a GPU here."""
import ctypes
import os
import re

import pytest

from paper_1205_2288_gb300 import tsbts

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include",
                      "tsbts.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tsbts_[a-z_]+)\s*\(", text)))


def test_header_lists_match_binding():
    assert declared_functions() == sorted(tsbts.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = tsbts.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_version_and_defaults():
    assert "sm_103a" in tsbts.tsbts_version()
    cfg = tsbts.tsbts_config_default()
    assert (cfg.precision, cfg.n_iter, cfg.era_mode, cfg.era_log2) == (0, 3, 0, 3)
    assert (cfg.k_max, cfg.exact_order, cfg.graph_steps) == (20, -1, 32)


def test_config_validation_happens_before_device_use():
    bad = tsbts.tsbts_config_default()
    bad.n_iter = 0
    with pytest.raises(tsbts.TsbtsError) as e:
        tsbts.tsbts_create(bad)
    assert e.value.code == tsbts.TSBTS_ERR_ARG
    bad = tsbts.tsbts_config_default()
    bad.graph_steps = 3          # graph steps come in slot pairs
    with pytest.raises(tsbts.TsbtsError) as e:
        tsbts.tsbts_create(bad)
    assert e.value.code == tsbts.TSBTS_ERR_ARG


def test_no_cpu_fallback_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(tsbts.TsbtsError) as e:
        tsbts.tsbts_create(tsbts.tsbts_config_default())
    assert e.value.code == tsbts.TSBTS_ERR_CUDA


def test_force_rejects_bad_arguments_without_touching_the_device():
    lib = tsbts.lib()
    assert lib.tsbts_force(5, -1, 10, 1, 1, 1, 0.0, 1, 1, 1, 1, 1, None) == -1
    assert lib.tsbts_force(0, -1, 0, 1, 1, 1, 0.0, 1, 1, 1, 1, 1, None) == -1
    assert lib.tsbts_force(0, -1, 10, 1, 1, 1, -1.0, 1, 1, 1, 1, 1, None) == -1
    assert lib.tsbts_force(0, -1, 10, 1, 1, 1, 0.0, -3, 1, 1, 1, 1, None) == -1
    assert lib.tsbts_force(0, -1, 10, 1, 1, 1, 0.0, 0, None, None, None,
                           None, None) == 0
