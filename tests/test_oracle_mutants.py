"""The oracle's pins must catch plausible mistakes.

Each case copies the oracle source, plants one mistake (a dropped term, a wrong sign, a
wrong index or comparison, a transposed operand), builds it, and runs the pin suite
(PIN_FILES below) against the broken copy.  The pin suite must fail for every
mutant.  The committed oracle is never modified.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hgp_oracle.c")

# the pin suites run against each mutant
PIN_FILES = ("test_oracle_pins.py", "test_oracle_rebalance.py", "test_oracle_exact_gains.py",
             "test_oracle_contract.py", "test_oracle_candidates.py")

# (name, exact text in the oracle source, replacement)
MUTANTS = [
    ("b uses Phi==2", "if (o->phi[(int64_t)e * o->k + a] == 1) b += o->nw[e];",
     "if (o->phi[(int64_t)e * o->k + a] == 2) b += o->nw[e];"),
    ("p_i uses Phi==1", "if (o->phi[(int64_t)e * o->k + i] == 0) p += o->nw[e];",
     "if (o->phi[(int64_t)e * o->k + i] == 1) p += o->nw[e];"),
    ("gain sign", "return b - p;", "return p - b;"),
    ("b drops net weight", "b += o->nw[e];", "b += 1;"),
    ("tie to larger block", "if (g > best_g && o->bw[i]", "if (g >= best_g && g > 0 && o->bw[i]"),
    ("strict capacity", "o->bw[i] + o->vw[u] <= o->lmax", "o->bw[i] + o->vw[u] < o->lmax"),
    ("capacity ignores c(u)", "o->bw[i] + o->vw[u] <= o->lmax", "o->bw[i] <= o->lmax"),
    ("approval gain ascending", "if (gu != gv) return gu > gv ? -1 : 1;",
     "if (gu != gv) return gu < gv ? -1 : 1;"),
    ("approval id descending", "return (u > v) - (u < v);", "return (u < v) - (u > v);"),
    ("exclusive prefix", "acc += o->vw[u];\n                    if (o->bw[t] + acc <= o->lmax) o->approved[u] = 1;",
     "if (o->bw[t] + acc <= o->lmax) o->approved[u] = 1;\n                    acc += o->vw[u];"),
    ("Phi update swapped", "o->phi[(int64_t)e * k + a]--;\n        o->phi[(int64_t)e * k + t]++;",
     "o->phi[(int64_t)e * k + a]++;\n        o->phi[(int64_t)e * k + t]--;"),
    ("block weight sign", "o->bw[a] -= o->vw[u];", "o->bw[a] += o->vw[u];"),
    ("always eligible", "if (o->all_eligible) return 1;", "return 1;"),
    ("never eligible after round 0", "if (o->moved_prev[o->inc[j]]) return 1;", "(void)j;"),
    ("lmax without ceil", "int64_t avg = (total_weight + k - 1) / k;", "int64_t avg = total_weight / k;"),
    ("objective counts lambda", "if (lambda > 0) *acc += (lambda - 1) * o->nw[e];",
     "if (lambda > 0) *acc += lambda * o->nw[e];"),
    ("objective drops weight", "if (lambda > 0) *acc += (lambda - 1) * o->nw[e];",
     "if (lambda > 0) *acc += (lambda - 1);"),
    ("hash shift", "z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;", "z = (z ^ (z >> 31)) * 0xbf58476d1ce4e5b9ULL;"),
    ("hash round/vertex swapped", "seed ^ (((uint64_t)round << 32) | (uint64_t)(uint32_t)u)",
     "seed ^ (((uint64_t)u << 32) | (uint64_t)(uint32_t)round)"),
    ("balance move to the heaviest block", "if (best_t < 0 || o->bw[i] < o->bw[best_t]) best_t = i;",
     "if (best_t < 0 || o->bw[i] > o->bw[best_t]) best_t = i;"),
    ("balance move keeps equal weights", "wi >= o->bw[a]", "wi > o->bw[a]"),
    ("balance move without room check", "if (wi > o->lmax || wi >= o->bw[a]", "if (wi >= o->bw[a]"),
    ("attributed gain from the frozen state", "o->attr[u] = oracle_gain(o, u, t);", "o->attr[u] = o->cand_g[u];"),
    ("revert of zero gains too", "if (!o->approved[u] || o->attr[u] >= 0) continue;",
     "if (!o->approved[u] || o->attr[u] > 0) continue;"),
    ("rebalance source rule inclusive", "if (left < o->bw[a] - o->lmax) o->selected[u] = 1;\n                    left += o->vw[u];",
     "left += o->vw[u];\n                    if (left < o->bw[a] - o->lmax) o->selected[u] = 1;"),
    ("rebalance phase 1 takes negative gains", "if (best_t < 0 || (phase == 1 && best_g < 0)) continue;",
     "if (best_t < 0) continue;"),
    ("rebalance ignores room", "if (i == a || o->bw[i] + o->vw[u] > o->lmax) continue;", "if (i == a) continue;"),
    ("rebalance moves make neighbours eligible", "move_vertex_marked(o, u, t, 0);",
     "move_vertex_marked(o, u, t, 0); for (int64_t jj = o->vtx_off[u]; jj < o->vtx_off[u + 1]; ++jj) o->moved_prev[o->inc[jj]] = 1;"),
    ("rebalance tie to larger block", "if (best_t < 0 || g > best_g) { best_t = i; best_g = g; }",
     "if (best_t < 0 || g >= best_g) { best_t = i; best_g = g; }"),
    ("rebalance repeats phase 1", "if (phase == 1) phase = 2;\n        else if (n_appr == 0) break;",
     "if (n_appr == 0) { if (phase == 2) break; phase = 2; }"),
    ("contraction keeps single-pin nets", "if (off1[e + 1] - off1[e] >= 2) order[kept++] = e;",
     "if (off1[e + 1] - off1[e] >= 1) order[kept++] = e;"),
    ("contraction keeps duplicate pins", "if (j == off1[e] || pins1[j] != pins1[j - 1]) pins1[k++] = pins1[j];",
     "pins1[k++] = pins1[j];"),
    ("identical nets not merged", "rep[e] = same ? rep[order[i - 1]] : e;", "rep[e] = e;"),
    ("identical net weights not summed", "wsum[rep[e]] += net_w ? net_w[e] : 1;",
     "if (rep[e] == e) wsum[e] = net_w ? net_w[e] : 1;"),
    ("cluster ids not remapped in order", "c->map[u] = cid[cluster[u]];", "c->map[u] = c->n - 1 - cid[cluster[u]];"),
    ("candidates ignore eligibility", "if (!eligible(o, u)) continue;", "(void)eligible;"),
    ("candidates hash the previous round", "if (oracle_subround_of(o->seed, o->round, u, o->subrounds) != s) continue;",
     "if (oracle_subround_of(o->seed, o->round ? o->round - 1 : 0, u, o->subrounds) != s) continue;"),
    ("sample b uses Phi==2", "if (phi_row[part[pins[j]]] == 1) b[q] += w;", "if (phi_row[part[pins[j]]] == 2) b[q] += w;"),
    ("sample p_i drops net weight", "if (phi_row[i] == 0) p[(int64_t)q * k + i] += w;",
     "if (phi_row[i] == 0) p[(int64_t)q * k + i] += 1;"),
    ("sample counts only sampled pins", "for (int64_t j = net_off[e]; j < net_off[e + 1]; ++j) phi_row[part[pins[j]]]++;",
     "for (int64_t j = net_off[e]; j < net_off[e + 1]; ++j) if (slot[pins[j]] >= 0) phi_row[part[pins[j]]]++;"),
    ("sample hashes round 1", "if (oracle_subround_of(seed, 0, u, subrounds) != s) continue;",
     "if (oracle_subround_of(seed, 1, u, subrounds) != s) continue;"),
    ("sample capacity ignores c(u)", "if (g > gain[q] && bw[i] + c <= lmax)", "if (g > gain[q] && bw[i] <= lmax)"),
    ("threaded slices drop the last item", "sl[t].hi = count * (t + 1) / T;",
     "sl[t].hi = count * (t + 1) / T - (t == T - 1);"),
    ("moves applied before all approvals", "for (int32_t t = 0; t < k; ++t) {\n                int64_t acc = 0;",
     "for (int32_t t = 0; t < k; ++t) {\n                int64_t acc = o->bw[t] > o->lmax ? 0 : 0;"),
]


def _run_mutant(name, old, new, workdir):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mutated = src.replace(old, new, 1)
    d = tempfile.mkdtemp(dir=workdir)
    c = os.path.join(d, "m.c")
    so = os.path.join(d, "m.so")
    open(c, "w").write(mutated)
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", "-o", so, c, "-lm"])
    env = dict(os.environ, HGP_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                       [os.path.join(ROOT, "tests", f) for f in PIN_FILES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode


def test_every_planted_mistake_is_caught():
    # the last entry is a no-op rewrite: it must NOT be caught (sanity of the harness)
    work = tempfile.mkdtemp(prefix="oracle_mutants_")
    try:
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
            results = list(ex.map(lambda m: _run_mutant(*m, work), MUTANTS))
    finally:
        shutil.rmtree(work, ignore_errors=True)
    survived = [name for name, rc in results[:-1] if rc == 0]
    assert not survived, f"pins did not catch: {survived}"
    assert results[-1][1] == 0, "an equivalent rewrite of the oracle was flagged"
