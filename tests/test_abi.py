"""The C ABI without a GPU: the library builds, loads, exports every symbol that
include/*.h declares, and rejects bad descriptors and arguments synchronously."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_2008_08483_gb300 import build as B
from paper_2008_08483_gb300 import chem, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return chem.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(chem_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "chem_source_term" in names and "chem_mechanism_load" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_abi_version(lib):
    text = open(os.path.join(ROOT, "include", "chem.h")).read()
    v = int(re.search(r"#define CHEM_ABI_VERSION (\d+)", text).group(1))
    assert chem.abi_version() == v


def _load_status(mech):
    try:
        chem.Mechanism(mech)
    except chem.ChemError as e:
        return e.status, str(e)
    return 0, ""


@pytest.mark.parametrize("mutate,needle", [
    (lambda m: m.nu_f.__setitem__((3, 0), m.nu_f[3, 0] + 1), "not balanced"),
    (lambda m: m.nu_f.__setitem__((2, 1), -1), "coefficient"),
    (lambda m: m.mol_weight.__setitem__(0, 0.0), "mol_weight"),
    (lambda m: m.kind.__setitem__(0, 7), "kind"),
    (lambda m: m.reversible.__setitem__(0, 2), "reversible"),
    (lambda m: m.arrh.__setitem__((1, 0), np.nan), "Arrhenius"),
    (lambda m: m.nasa7.__setitem__((1, 0, 0), np.inf), "nasa7"),
    (lambda m: setattr(m, "t_mid", -1.0), "t_mid"),
    (lambda m: setattr(m, "p_ref", 0.0), "p_ref"),
])
def test_descriptor_validation(lib, mutate, needle):
    m = synth.make_mechanism("h2air_9_21", seed=1).copy()
    mutate(m)
    st, msg = _load_status(m)
    assert st == 1 and needle in msg, msg


def test_troe_validation(lib, mech53):
    m = mech53.copy()
    j = int(np.nonzero(m.kind == 3)[0][0])
    m.troe[j, 1] = 0.0
    st, msg = _load_status(m)
    assert st == 1 and "Troe" in msg


def test_source_term_argument_errors(lib):
    L = lib
    P = C.c_void_p
    assert L.chem_source_term(None, 1, P(8), P(8), P(8), 9, P(8), 9, 0, None) == 1
    assert b"NULL" in L.chem_last_error()
    assert L.chem_mechanism_load(None, C.byref(P())) == 1
    assert L.chem_mechanism_free(None) == 0
