"""Register and spill budgets of the timed kernels, from ptxas' resource
report of the in-tree build (no GPU).  Each budget is the one the kernel's
launch bounds were chosen for: a change that makes a kernel spill, or pushes
it past the registers its resident blocks per SM allow, shows up here before
it shows up as a slower step."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BUILD = os.path.join(ROOT, "paper_1909_04502_gb300", "_build")


@pytest.fixture(scope="module")
def reports():
    import shutil
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_1909_04502_gb300 import build
    build.build()
    out = {}
    for name in os.listdir(BUILD):
        if name.endswith(".ptxas.txt"):
            out[name.split(".")[0]] = open(os.path.join(BUILD, name)).read()
    return out


def _entries(txt):
    """{mangled kernel name: (registers, spill store bytes, spill load bytes)}"""
    res = {}
    blocks = re.split(r"ptxas info\s+: Compiling entry function '", txt)[1:]
    for b in blocks:
        name = b.split("'", 1)[0]
        regs = re.search(r"Used (\d+) registers", b)
        sp = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", b)
        if regs and sp:
            res[name] = (int(regs.group(1)), int(sp.group(1)), int(sp.group(2)))
    return res


def _find(entries, pattern):
    hits = {k: v for k, v in entries.items() if re.search(pattern, k)}
    assert hits, pattern
    return hits


# (source, mangled-name pattern, register budget, spill-store budget in bytes)
BUDGETS = [
    # the headline step: FP32 storage, Q = 28, bilinear, orbit-symmetric (seven blocks per SM)
    ("step_o2", r"k_stepIfLi28ELb1ELi9ELi1ELb1ELb0ELb0E", 72, 0),
    # the same, on-lattice (eight blocks per SM)
    ("step_o2", r"k_stepIfLi28ELb1ELi9ELi0ELb1ELb0ELb0E", 64, 0),
    # force / walls on the orbit-symmetric path, on-lattice (six blocks per SM)
    ("step_o2", r"k_stepIfLi29ELb1ELi9ELi0ELb1ELb0ELb1E", 80, 0),
    # order 3, orbit-symmetric, Q = 49 (six blocks per SM) and Q = 65 (five)
    ("step_o3m", r"k_stepIfLi49ELb1ELi16ELi0ELb1ELb0ELb0E", 80, 0),
    ("step_o3m", r"k_stepIfLi65ELb1ELi16ELi0ELb1ELb0ELb0E", 96, 0),
    # (3+1)-d FP32 steps in sign-orbit form
    ("step3", r"k_step3fs", 64, 16),
    ("step3q", r"k_step3qsf", 80, 0),
    # (1+1)-d FP32 step, order 3, two cells per thread
    ("d1", r"k_step1fILi3ELi2E", 64, 0),
]


@pytest.mark.parametrize("src,pattern,regs,spill", BUDGETS)
def test_kernel_stays_within_its_register_and_spill_budget(reports, src, pattern, regs, spill):
    for name, (r, st, ld) in _find(_entries(reports[src]), pattern).items():
        assert r <= regs, (name, r)
        assert st <= spill and ld <= spill, (name, st, ld)
