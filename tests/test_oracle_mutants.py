"""How strong the oracle's pins are: plausible mistakes planted in copies of
the oracle's sources must each fail at least one pin.

Each mutant below is a small edit of oracle.cpp or kl_frontend.hpp (a dropped
term, a flipped comparison, a wrong index or witness, a rule read the wrong
way).  The copy is compiled on the CPU into its own library and
tests/test_oracle_pins.py runs against it in a child process (the oracle
wrapper loads the library named by RC_ORACLE_LIB).  A mutant the pins let
through would be a mistake the oracle could make unseen.  The unmutated copy,
built the same way, must pass, so that a failure is the planted mistake's and
not the harness's.

The explorer (explore.cpp) is a pin itself and is not mutated; the front end
it shares with the oracle is, so front-end mutants must be caught by pins that
do not go through the explorer (goldens, closed forms, arithmetic tables).
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")
PINS = os.path.join("tests", "test_oracle_pins.py")

# name -> (file, [(original text, replacement)]); every original occurs once.
MUTANTS = {
    "control": ("oracle.cpp", []),
    # Sec. 4 race rule, write/write: the interval's final value is each
    # writer's last write; comparing first writes misses overwritten values.
    "ww_compares_first_writes": ("oracle.cpp", [
        ("int32_t l1 = writes.begin()->second.back();", "int32_t l1 = writes.begin()->second.front();"),
        ("if (w.second.back() != l1) { race = true;", "if (w.second.front() != l1) { race = true;"),
    ]),
    # the benign rule dropped: any two writers race whatever they write
    "ww_benign_rule_dropped": ("oracle.cpp", [
        ("if (w.second.back() != l1) { race = true;", "if (w.first != w1) { race = true;"),
    ]),
    "ww_witness_is_largest_writer": ("oracle.cpp", [
        ("if (race) { r.cls = C_WW_RACE; r.t_a = w1; r.t_b = tb; }",
         "if (race) { r.cls = C_WW_RACE; r.t_a = w1; r.t_b = writes.rbegin()->first; }"),
    ]),
    # a work-item's read of its own write counted as a conflict
    "rw_self_conflict": ("oracle.cpp", [
        ("if (w.first == rd.first) continue;", ""),
    ]),
    # a writer of several values agrees with a reader that saw one of them
    "rw_ignores_other_written_values": ("oracle.cpp", [
        ("bool same = obs.size() == 1 && w.second.size() == 1 && *obs.begin() == *w.second.begin();",
         "bool same = obs.size() == 1 && w.second.count(*obs.begin()) == 1;"),
    ]),
    "rw_witness_reader_writer_swapped": ("oracle.cpp", [
        ("r.t_a = best_r;\n        r.t_b = best_j;", "r.t_a = best_j;\n        r.t_b = best_r;"),
    ]),
    "counts_readers_writers_swapped": ("oracle.cpp", [
        ("(uint32_t)reads.size(), (uint32_t)writes.size(), (uint32_t)acc.size()}",
         "(uint32_t)writes.size(), (uint32_t)reads.size(), (uint32_t)acc.size()}"),
    ]),
    # delayed visibility: a read no longer sees the work-item's own write
    "read_ignores_own_write": ("oracle.cpp", [
        ("int32_t v = it != own.end() ? it->second : committed(c);", "int32_t v = committed(c);"),
    ]),
    # commit: the lowest writer instead of the highest
    "commit_lowest_writer": ("oracle.cpp", [
        ("if (a.write && (!any || a.gtid > top)) { top = a.gtid; any = true; }",
         "if (a.write && (!any || a.gtid < top)) { top = a.gtid; any = true; }"),
    ]),
    # commit: the top writer's first write instead of its last
    "commit_first_write_of_top_writer": ("oracle.cpp", [
        ("if (a.write && a.gtid == top) v = a.value;", "if (a.write && a.gtid == top) { v = a.value; break; }"),
    ]),
    # Table 1 bounds premise off by one
    "oob_bound_off_by_one": ("oracle.cpp", [
        ("if (idx < 0 || (int64_t)idx >= mem_len[n.mem]) {", "if (idx < 0 || (int64_t)idx > mem_len[n.mem]) {"),
    ]),
    # barrier-release rule: exited work-items not counted as a stop point
    "exit_not_a_stop_point": ("oracle.cpp", [
        ("else if (th[g].st == EXITED) id = 0xFFFFFFFFu;\n        else continue;\n        auto it = stops.find(id);\n"
         "        if (it == stops.end()) stops[id] = {g, 1};\n        else it->second.second++;\n      }\n      bool diverged",
         "else continue;\n        auto it = stops.find(id);\n"
         "        if (it == stops.end()) stops[id] = {g, 1};\n        else it->second.second++;\n      }\n      bool diverged"),
    ]),
    # assume(b) with b false taken as a no-op instead of ending the path
    "assume_ignored": ("oracle.cpp", [
        ("if (eval(*n.val, env) == 0) { t.st = DEAD; return; }  // ⊤", "(void)0;"),
    ]),
    # a failed assert records nothing
    "assert_silent": ("oracle.cpp", [
        ("errors.push_back({interval, 0, 0, 0, C_ASSERT, gtid, (uint32_t)n.id, 0, 0, 0});", ""),
    ]),
    # front end: the else edge guarded by the condition itself, not its negation
    "else_guard_not_negated": ("kl_frontend.hpp", [
        ("Node f{N_ASSUME};\n        f.val = negate(b);", "Node f{N_ASSUME};\n        f.val = b;"),
    ]),
    # local memory shared by all work-groups
    "local_memory_not_per_group": ("oracle.cpp", [
        ("Cell c{(uint32_t)m.space, m.space ? wg : 0u, (uint32_t)(mem_base[n.mem] + (uint64_t)idx)};",
         "Cell c{(uint32_t)m.space, 0u, (uint32_t)(mem_base[n.mem] + (uint64_t)idx)};"),
    ]),
    # group scope: the value before the run left out of "held one value all along"
    "xg_ignores_initial_value": ("oracle.cpp", [
        ("all.insert(initial_global[kv.first]);", ""),
    ]),
    # group scope: witness rule compares work-items instead of their groups
    "xg_witness_compares_items": ("oracle.cpp", [
        ("if (r0 / S != w0 / S) { r.t_a = r0; r.t_b = w0; }", "if (r0 != w0) { r.t_a = r0; r.t_b = w0; }"),
    ]),
    # group scope: writers in one group counted as cross-group
    "xg_ww_within_one_group": ("oracle.cpp", [
        ("if (wgw.size() >= 2) {", "if (nwr >= 2) {"),
    ]),
    # address sharding: another shard's global cell commits its lowest writer
    "shard_pending_lowest_writer": ("oracle.cpp", [
        ("if (pend_writer[addr] == 0xFFFFFFFFu || gtid >= pend_writer[addr]) {",
         "if (pend_writer[addr] == 0xFFFFFFFFu || gtid <= pend_writer[addr]) {"),
    ]),
    # group scope: exited work-items not a stop point of their group
    "xg_exit_not_a_group_stop_point": ("oracle.cpp", [
        ("else if (th[g].st == EXITED) id = 0xFFFFFFFFu;  // exited in this round: the group was not done", ""),
    ]),
    # error records of one interval ordered by work-item before kind
    "errors_ordered_by_item_first": ("oracle.cpp", [
        ("return std::tie(a.cls, a.t_a) < std::tie(b.cls, b.t_a);", "return std::tie(a.t_a, a.cls) < std::tie(b.t_a, b.cls);"),
    ]),
    # loads left out of the access counter
    "loads_not_counted": ("oracle.cpp", [
        ("          rep.n_access++;\n", "          if (n.kind == N_STORE) rep.n_access++;\n"),
    ]),
    # front end: `%` truncating like C instead of Euclidean
    "mod_truncates": ("kl_frontend.hpp", [
        ("if (r < 0) r += m;", ""),
    ]),
    "le_is_lt": ("kl_frontend.hpp", [
        ("case E_LE: { int32_t x = A(), y = B(); return x <= y; }",
         "case E_LE: { int32_t x = A(), y = B(); return x < y; }"),
    ]),
    # front end: `for v in lo .. hi` running hi inclusive
    "for_bound_inclusive": ("kl_frontend.hpp", [
        ("cond->kind = E_LT;", "cond->kind = E_LE;"),
    ]),
    # front end: global id from the group count instead of the group size
    "gtid_uses_group_count": ("kl_frontend.hpp", [
        ("(uint64_t)env.wg * env.gsize + env.tid", "(uint64_t)env.wg * env.ngroups + env.tid"),
    ]),
    # front end: division by zero not caught (yields the dividend)
    "div_by_zero_yields_dividend": ("kl_frontend.hpp", [
        ("      if (y == 0) return 0;\n      return (int32_t)(uint32_t)(uint64_t)(x / y);",
         "      if (y == 0) return (int32_t)x;\n      return (int32_t)(uint32_t)(uint64_t)(x / y);"),
    ]),
}


def _build(name, workdir):
    fname, edits = MUTANTS[name]
    d = os.path.join(workdir, name)
    os.makedirs(d)
    for f in ("oracle.cpp", "explore.cpp", "kl_frontend.hpp"):
        shutil.copy(os.path.join(ORACLE_DIR, f), d)
    path = os.path.join(d, fname)
    text = open(path, encoding="utf-8").read()
    for old, new in edits:
        assert text.count(old) == 1, (name, old)
        text = text.replace(old, new)
    open(path, "w", encoding="utf-8").write(text)
    lib = os.path.join(d, "liboracle.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", lib, "oracle.cpp", "explore.cpp"],
                   check=True, cwd=d, capture_output=True)
    return lib


def _pins(lib, select):
    env = dict(os.environ, RC_ORACLE_LIB=lib)
    p = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", "-k", select],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout[-2000:]


def _run(name, workdir):
    lib = _build(name, workdir)
    if name == "control":  # the slow brute-force pins run in the main suite already
        return _pins(lib, "not bruteforce")
    rc, out = _pins(lib, "not bruteforce")
    if rc == 0:
        rc, out = _pins(lib, "bruteforce")
    return rc, out


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    workdir = str(tmp_path_factory.mktemp("oracle_mutants"))
    names = sorted(MUTANTS)
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda n: _run(n, workdir), names))
    return dict(zip(names, results))


def test_unmutated_copy_passes_the_pins(outcomes):
    rc, out = outcomes["control"]
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(n for n in MUTANTS if n != "control"))
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, out = outcomes[name]
    # 1: some pin failed (2-5 would be an interrupted run or a harness error)
    assert rc == 1, (name, rc, out)
    assert " failed" in out, out


# ---- the ranking network's reference (oracle/mlp_ref.py) against its pins
# (tests/test_mlp_ref.py: finite differences, closed forms, torch's bfloat16
# rounding)
MLP_MUTANTS = {
    "control": [],
    "relu_derivative_always_one": [('dz = rnd(np.outer(dl, c["w4"]) * (c["h"][3] > 0))',
                                    'dz = rnd(np.outer(dl, c["w4"]) * (c["h"][3] >= 0))')],
    "backward_through_transposed_weights": [('dz = rnd((dz @ c["W"][l]) * (c["h"][l] > 0))',
                                             'dz = rnd((dz @ c["W"][l].T) * (c["h"][l] > 0))')],
    "bias_gradient_averaged_twice": [('g[f"b{l + 1}"] = dz.sum(axis=0)', 'g[f"b{l + 1}"] = dz.mean(axis=0)')],
    "weight_gradient_from_wrong_layer": [('g = {"w4": dl @ c["h"][3]', 'g = {"w4": dl @ c["h"][2]')],
    "loss_without_softplus_term": [("loss = np.mean(np.maximum(z, 0) + np.log1p(np.exp(-np.abs(z))) - y * z)",
                                    "loss = np.mean(np.maximum(z, 0) - y * z)")],
    "sigmoid_sign_flipped": [("prob = 1.0 / (1.0 + np.exp(-z))", "prob = 1.0 / (1.0 + np.exp(z))")],
    "output_bias_dropped": [('z = hs[3] @ w4 + np.asarray(P["b4"], dtype=dtype)[0]', "z = hs[3] @ w4")],
    "bf16_ties_away_from_zero": [("u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "u = (u + 0x8000) & 0xFFFF0000")],
    "hidden_activation_not_rounded": [("hs.append(rnd(np.maximum(z, 0)))", "hs.append(np.maximum(z, 0))")],
    "adam_first_moment_not_decayed": [("m = b1 * m + (1.0 - b1) * g", "m = m + (1.0 - b1) * g")],
    "adam_bias_corrections_swapped": [("m_hat = m / (1.0 - b1 ** t)", "m_hat = m / (1.0 - b2 ** t)")],
    "adam_eps_inside_the_root": [("p - lr * m_hat / (np.sqrt(v_hat) + eps)", "p - lr * m_hat / np.sqrt(v_hat + eps)")],
    "adam_correction_one_step_late": [("v_hat = v / (1.0 - b2 ** t)", "v_hat = v / (1.0 - b2 ** (t + 1))")],
}

MLP_CHILD = ("import importlib.util, sys\n"
             "import oracle\n"
             "spec = importlib.util.spec_from_file_location('oracle.mlp_ref', sys.argv[1])\n"
             "m = importlib.util.module_from_spec(spec)\n"
             "spec.loader.exec_module(m)\n"
             "sys.modules['oracle.mlp_ref'] = m\n"
             "oracle.mlp_ref = m\n"
             "import pytest\n"
             "sys.exit(pytest.main(sys.argv[2:]))\n")


def _mlp_run(name, workdir):
    text = open(os.path.join(ORACLE_DIR, "mlp_ref.py"), encoding="utf-8").read()
    for old, new in MLP_MUTANTS[name]:
        assert text.count(old) == 1, (name, old)
        text = text.replace(old, new)
    path = os.path.join(workdir, f"mlp_ref_{name}.py")
    open(path, "w", encoding="utf-8").write(text)
    p = subprocess.run([sys.executable, "-c", MLP_CHILD, path, os.path.join("tests", "test_mlp_ref.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout[-2000:]


@pytest.fixture(scope="module")
def mlp_outcomes(tmp_path_factory):
    workdir = str(tmp_path_factory.mktemp("mlp_mutants"))
    names = sorted(MLP_MUTANTS)
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda n: _mlp_run(n, workdir), names))
    return dict(zip(names, results))


def test_unmutated_network_reference_passes(mlp_outcomes):
    rc, out = mlp_outcomes["control"]
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(n for n in MLP_MUTANTS if n != "control"))
def test_planted_network_mistake_fails_a_pin(mlp_outcomes, name):
    rc, out = mlp_outcomes[name]
    assert rc == 1, (name, rc, out)
    assert " failed" in out, out
