"""The C ABI library loads and exports every symbol its headers declare (CPU only).

No compute entry point is called here: this box may have no GPU.
"""
import ctypes
import glob
import os
import re

import pytest

from paper_2209_04015_b300 import build as libbuild
from paper_2209_04015_b300 import afqmc as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(afq_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return binding.load_library()


def test_headers_declare_the_boundary():
    names = declared_symbols()
    for core in ("afq_init_hamiltonian", "afq_init_trial", "afq_init_walkers", "afq_propagate",
                 "afq_local_energy", "afq_orthogonalise"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_c_names(lib):
    names = declared_symbols()
    for n in names:
        short = n[len("afq_"):]
        if short in ("create", "destroy", "last_error", "default_params", "kernel_name"):
            continue
        if short.startswith("batch_"):
            sub = short[len("batch_"):]
            assert sub in ("create", "destroy", "last_error") or hasattr(binding.AfqBatch, sub), short
            continue
        assert hasattr(binding.AfqContext, short) or hasattr(binding, short), short


def test_default_params_are_host_only(lib):
    p = binding.AfqParams()
    lib.afq_default_params(ctypes.byref(p))
    assert p.dt == 0.005 and p.taylor_order == 6 and p.qr_period == 5 and p.seed == 1
    assert p.precision == 0 and p.fb_cap == 0.0 and p.free_projection == 0
    assert p.exchange == binding.EXCHANGES["auto"]
    assert lib.afq_last_error(None) == b"null context"


def test_null_context_is_rejected_without_touching_the_gpu(lib):
    assert lib.afq_destroy(None) == binding.AFQ_ERR_ARG
    assert lib.afq_propagate(None, None, 1) == binding.AFQ_ERR_ARG
    assert lib.afq_create(None, None, None) == binding.AFQ_ERR_ARG
