"""Static check of bench.py and __graft_entry__.py: every name a function
reads that is not local or enclosing must exist at module level or in
builtins (the benchmark only runs on a GPU, so a stale name would otherwise
surface only there)."""
import builtins
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _unresolved(path):
    src = open(path).read()
    top = symtable.symtable(src, path, "exec")
    defined = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported() or s.is_namespace()}
    defined |= set(dir(builtins))
    bad = []

    def walk(t):
        for c in t.get_children():
            if c.get_type() == "function":
                for s in c.get_symbols():
                    if s.is_referenced() and s.is_global() and s.get_name() not in defined:
                        bad.append((c.get_name(), s.get_name()))
            walk(c)

    walk(top)
    return bad


@pytest.mark.parametrize("name", ["bench.py", "__graft_entry__.py"])
def test_no_unresolved_names(name):
    assert _unresolved(os.path.join(ROOT, name)) == []
