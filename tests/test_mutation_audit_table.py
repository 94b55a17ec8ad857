"""The mutation audit (tests/mutation_audit.py) stays runnable: every planted mistake still applies to
exactly one place of the current sources, and changes it."""
import os

import pytest

from mutation_audit import HOST_MUTANTS, MUTANTS, ROOT

ALL = [("oracle",) + m for m in MUTANTS] + [("host",) + m for m in HOST_MUTANTS]


@pytest.mark.parametrize("table,name,path,old,new", ALL, ids=[m[0] + ":" + m[1] for m in ALL])
def test_mutant_applies_once(table, name, path, old, new):
    assert path.startswith("oracle/") if table == "oracle" else path.endswith("csrc/tc_setup.cpp")
    text = open(os.path.join(ROOT, path)).read()
    assert text.count(old) == 1, name
    assert old != new


def test_mutant_names_are_unique():
    names = [m[1] for m in ALL]
    assert len(names) == len(set(names))
