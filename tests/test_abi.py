"""The C-ABI library loads and exports every entry point include/colapm.h declares (no GPU calls)."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))
LIB = os.path.join(ROOT, "paper_1506_03737_gb300", "_lib", "libcolapm.so")


def declared():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(colapm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1506_03737_gb300 import build
        build.build()
    from paper_1506_03737_gb300 import colapm
    return colapm


def test_header_declares_the_boundary():
    names = declared()
    for must in ("colapm_create", "colapm_make_ics", "colapm_step", "colapm_power", "colapm_destroy",
                 "colapm_nn_create", "colapm_nn_train_step", "colapm_nn_forward", "colapm_get_displacement"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib.LIB, n)]
    assert not missing, missing


def test_params_struct_and_defaults(lib):
    import ctypes
    p = lib.default_params()
    assert ctypes.sizeof(p) == 5 * 8 + 8 + 4 + 4 + 8 + 8 + 4 + 4 + 4 + 4 + 8 + 4 + 4 + 8
    assert (p.np, p.nm, p.n_steps, p.cola, p.deconv) == (32, 64, 10, 1, 1)
    assert p.nlpt == -2.5 and p.cosmo.sigma8 == 0.8
    assert lib.strerror(-4) == "fixed-point density overflow"


def test_nn_config_struct_and_defaults(lib):
    import ctypes
    c = lib.nn_default_config()
    assert ctypes.sizeof(c) == 6 * 4 + 4 + 4 + 8          # int engine, padding, u64 seed
    assert c.engine == 0
    assert (c.lr, c.beta1, c.eps, c.seed) == (np.float32(1e-3), np.float32(0.9), np.float32(1e-8), 1)
    assert lib.NN_PARAMS == 16467
