"""The mutation audit of the oracle's pins (tests/oracle_mutants.py) stays runnable: every planted
mistake still applies to exactly one place of the current oracle sources, and changes it."""
import os

import pytest

from oracle_mutants import MUTANTS, ROOT


@pytest.mark.parametrize("name,path,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_applies_once(name, path, old, new):
    assert path.startswith("oracle/")
    text = open(os.path.join(ROOT, path)).read()
    assert text.count(old) == 1, name
    assert old != new


def test_mutant_names_are_unique():
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))
