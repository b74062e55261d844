"""How strong the host-side tests of the library are: mistakes planted in
copies of prove.cpp must each fail tests/test_prove_cpu.py, and mistakes
planted in copies of translate.cpp must each fail tests/test_translate_cpu.py.

The pre-filter's claims (race freedom, bounds, private accesses) are
one-sided: an unsound claim would let the checker skip logging an access or
declare an instance race-free that is not.  Each mutant below widens what
the analysis claims (an off-by-one in a range or a guard, a check left out, a
loop counter range cut short, a pair cleared by the benign-value rule where
only cell disjointness may clear it).  The copy is compiled on the CPU and
linked with the library's other objects; the tests then run against it in
a child process.  The unmutated copies, built the same way, must pass them.

The translator's mutants are plausible slips in writing a bytecode
instruction as C++: a loop's back edge taken once more, operands of a
reversed subtraction or a multiply-add swapped, a branch condition of the
wrong sense, the resume point after a barrier, the constant part of an
index, a logical not of the wrong sense.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = {"prove.cpp": os.path.join("tests", "test_prove_cpu.py"),
         "translate.cpp": os.path.join("tests", "test_translate_cpu.py")}

MUTANTS = {
    "control": [],
    # two index ranges that touch at one cell taken as disjoint
    "disjoint_off_by_one": [("ok = ra.hi < rb.lo || rb.hi < ra.lo;", "ok = ra.hi <= rb.lo || rb.hi <= ra.lo;")],
    # equal index forms taken as one-to-one without the injectivity argument
    "same_form_is_one_to_one": [("ok = ok || (a.idx == b.idx && injective(a.idx, h, a.local));",
                                 "ok = ok || (a.idx == b.idx);")],
    # accesses of overlapping (not equal) barrier-region sets never paired
    "regions_must_be_equal": [("if (!(pr.region[a.pc] & pr.region[b.pc])) continue;",
                               "if (pr.region[a.pc] != pr.region[b.pc]) continue;")],
    # one tid per group taken as one work-item for a global array
    "one_tid_ignores_groups": [("(h.nt() == 1 && (a.local || h.nw() == 1))", "(h.nt() == 1)")],
    # a load reading back its own store stays private whoever else reads the cell
    "read_back_always_private": [("if (!store_pairs_clear[rr.second]) (*priv)[rr.first] = 0;", "")],
    # a `tid < k` guard admitting tid = k
    "guard_lt_inclusive": [("case 0: hi = cdiv(r, k) - 1; break;", "case 0: hi = cdiv(r, k); break;")],
    # a remainder taken as a plain shift across a period boundary
    "mod_range_ignores_period": [("if (fdiv(h, f.M) == q && l > -kSat && h < kSat)",
                                  "if (l > -kSat && h < kSat)")],
    # a one-to-one form taken as one-to-one after any reduction mod M
    "injective_ignores_modulus": [("return f.M == 0 || span < f.M;", "return true;")],
    # a loop counter's range one short at the top
    "loop_counter_range_short": [("sh.vhi[L] = std::max<int64_t>(lp.entry.c0, lp.hi - 1);",
                                  "sh.vhi[L] = std::max<int64_t>(lp.entry.c0, lp.hi - 2);")],
    # equal stored values clearing a pair for privacy, not only for race freedom
    "benign_values_clear_privacy": [
        ("if (!ok && priv) (*priv)[a.pc] = (*priv)[b.pc] = 0;  // the two may share a cell", ""),
        ("      if (!ok) {\n        if (out->race_free) {",
         "      if (!ok && priv) (*priv)[a.pc] = (*priv)[b.pc] = 0;\n      if (!ok) {\n        if (out->race_free) {"),
    ],
}

TRANSLATE_MUTANTS = {
    "translate_control": [],
    "loop_back_edge_inclusive": [('line(o, "  if (%s < %s) goto L%d;", d.c_str(), I.c_str(), imm2);',
                                  'line(o, "  if (%s <= %s) goto L%d;", d.c_str(), I.c_str(), imm2);')],
    "rsubi_operands_swapped": [
        ('case OP_RSUBI: line(o, "  %s = (int32_t)(%s%s - %s%s);", d.c_str(), U.c_str(), I.c_str(), U.c_str(), a.c_str());',
         'case OP_RSUBI: line(o, "  %s = (int32_t)(%s%s - %s%s);", d.c_str(), U.c_str(), a.c_str(), U.c_str(), I.c_str());')],
    "madi_operands_swapped": [
        ('line(o, "  %s = (int32_t)(%s%s * %s%s + %s%s);", d.c_str(), U.c_str(), a.c_str(), U.c_str(), I.c_str(),\n'
         '             U.c_str(), b.c_str());',
         'line(o, "  %s = (int32_t)(%s%s * %s%s + %s%s);", d.c_str(), U.c_str(), b.c_str(), U.c_str(), I.c_str(),\n'
         '             U.c_str(), a.c_str());')],
    "branch_ge_as_gt": [('case OP_BFGEI: return ">=";', 'case OP_BFGEI: return ">";')],
    "barrier_resumes_at_itself": [('line(o, "  RC_AT_BARRIER(cx, %d); pc = %u; st = %u; return;", imm, k + 1, (unsigned)TS_BARRIER);',
                                   'line(o, "  RC_AT_BARRIER(cx, %d); pc = %u; st = %u; return;", imm, k + 2, (unsigned)TS_BARRIER);')],
    "index_constant_dropped": [('"rc::sem_index(%s, %s, (int32_t)%" PRId32 "LL, %uu)", a.c_str(), I.c_str(), imm2,',
                                '"rc::sem_index(%s, %s, (int32_t)%" PRId32 "LL * 0, %uu)", a.c_str(), I.c_str(), imm2,')],
    "not_of_wrong_sense": [('case OP_NOT: line(o, "  %s = %s == 0;", d.c_str(), a.c_str()); break;',
                            'case OP_NOT: line(o, "  %s = %s != 0;", d.c_str(), a.c_str()); break;')],
}

CHILD = ("import sys\n"
         "import paper_1308_3203_gb300.racecheck as r\n"
         "r.LIB_PATH = sys.argv[1]\n"
         "import pytest\n"
         "sys.exit(pytest.main(sys.argv[2:]))\n")


def _target(name):
    return ("translate.cpp", TRANSLATE_MUTANTS[name]) if name in TRANSLATE_MUTANTS else ("prove.cpp", MUTANTS[name])


def _build(name, workdir, B):
    fname, edits = _target(name)
    d = os.path.join(workdir, name)
    os.makedirs(d)
    text = open(os.path.join(B.CSRC, fname), encoding="utf-8").read()
    for old, new in edits:
        assert text.count(old) == 1, (name, old)
        text = text.replace(old, new)
    src = os.path.join(d, fname)
    open(src, "w", encoding="utf-8").write(text)
    obj = os.path.join(d, fname.replace(".cpp", ".o"))
    nv = B._nvcc()
    subprocess.run([nv, "-x", "c++"] + B.NVFLAGS[len(B.ARCH):] + [f"-I{B.CSRC}", "-c", src, "-o", obj],
                   check=True, capture_output=True)
    objs = [os.path.join(B.OUT_DIR, os.path.splitext(s)[0] + ".o") for s in B.SOURCES if s != fname]
    lib = os.path.join(d, "libracecheck.so")
    subprocess.run([nv] + B.ARCH + ["-shared", "-o", lib, obj] + objs, check=True, capture_output=True)
    return lib


def _run(name, workdir, B):
    lib = _build(name, workdir, B)
    p = subprocess.run([sys.executable, "-c", CHILD, lib, TESTS[_target(name)[0]], "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    return p.returncode, p.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    from paper_1308_3203_gb300 import build as B
    objs = [os.path.join(B.OUT_DIR, os.path.splitext(s)[0] + ".o") for s in B.SOURCES]
    B.build(force=not all(os.path.exists(o) for o in objs))  # the other objects of the library
    workdir = str(tmp_path_factory.mktemp("prove_mutants"))
    names = sorted(MUTANTS) + sorted(TRANSLATE_MUTANTS)
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda n: _run(n, workdir, B), names))
    shutil.rmtree(workdir, ignore_errors=True)
    return dict(zip(names, results))


@pytest.mark.parametrize("name", ["control", "translate_control"])
def test_unmutated_copy_passes(outcomes, name):
    rc, out = outcomes[name]
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(n for n in list(MUTANTS) + list(TRANSLATE_MUTANTS) if "control" not in n))
def test_planted_mistake_fails_a_test(outcomes, name):
    rc, out = outcomes[name]
    assert rc == 1, (name, rc, out)
    assert " failed" in out, out
