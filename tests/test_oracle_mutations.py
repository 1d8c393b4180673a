"""The pins catch the oracle's plausible mistakes: each entry of `oracle_mutations.MUTATIONS` is
planted in a scratch copy of the oracle, and the pins of `test_oracle_pins.py` run against it;
at least one must fail (the equivalent entries, whose mistake changes nothing observable,
must pass).  Each entry builds and runs the pins once, a minute or two, so the check runs on
request only: EDAC_ORACLE_MUTATIONS=1 runs every entry, a comma-separated list of names runs
those (`python -m pytest tests/test_oracle_mutations.py -n 8` with pytest-xdist).  The
table itself is checked always: every text to replace occurs exactly once in the oracle."""
import os
import shutil
import subprocess
import sys

import pytest

from oracle_mutations import EQUIVALENT, MUTATIONS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "edac_oracle.c")


def _selected():
    sel = os.environ.get("EDAC_ORACLE_MUTATIONS", "")
    return sorted(MUTATIONS) if sel == "1" else sorted(n for n in sel.split(",") if n in MUTATIONS)


def test_every_planted_text_occurs_once_in_the_oracle():
    src = open(SRC).read()
    for name, pairs in MUTATIONS.items():
        for old, new in pairs:
            assert old != new, name
            assert src.count(old) == 1, (name, old)
    assert EQUIVALENT <= set(MUTATIONS)


@pytest.mark.slow
@pytest.mark.parametrize("name", _selected())
def test_planted_mistake_fails_a_pin(name, tmp_path):
    d = str(tmp_path)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                    ignore=shutil.ignore_patterns("_lib", "__pycache__"))
    os.makedirs(os.path.join(d, "tests"))
    for f in ("test_oracle_pins.py", "conftest.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
    os.makedirs(os.path.join(d, "paper_1907_04034_gb300"))
    for f in ("__init__.py", "cases.py"):
        shutil.copy(os.path.join(ROOT, "paper_1907_04034_gb300", f),
                    os.path.join(d, "paper_1907_04034_gb300", f))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    src_path = os.path.join(d, "oracle", "edac_oracle.c")
    src = open(src_path).read()
    for old, new in MUTATIONS[name]:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    open(src_path, "w").write(src)
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "2"))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                        "-p", "no:cacheprovider", "-m", "not slow"],
                       cwd=d, capture_output=True, text=True, env=env)
    failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED tests/test_oracle_pins.py")]
    if name in EQUIVALENT:
        assert r.returncode == 0, r.stdout[-2000:]
    else:
        # a pin fails (not a build or collection error)
        assert r.returncode == 1 and failed, (r.returncode, r.stdout[-2000:], r.stderr[-2000:])
