"""The oracle's pins fail plausible mistakes planted in a copy of it
(``oracle/mutants.py``: the full list runs with ``python -m oracle.mutants``;
here every mutation site is checked to exist once, and two mutants run)."""
from oracle import mutants


def test_every_mutation_site_is_found_once():
    src = open(mutants.SRC).read()
    names = [m[0] for m in mutants.MUTANTS]
    assert len(set(names)) == len(names)
    for name, find, replace, areas in mutants.MUTANTS:
        assert src.count(find) == 1, name
        assert find != replace and areas, name


def test_planted_mistakes_are_caught():
    res = mutants.run(["copy_from_no_zero_fill", "walk_fault_level_dropped"])
    assert res == {"copy_from_no_zero_fill": "killed", "walk_fault_level_dropped": "killed"}
