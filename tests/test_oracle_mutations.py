"""The oracle's pins are strong enough: each planted mistake makes at least one pin fail.

Every case below edits a copy of the oracle's C source (a dropped term, a flipped sign, a wrong
index, a transposed operand), compiles it on the CPU, and runs the pin suites against that build
in a child pytest process. The child run must fail. The shipped oracle is untouched.
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "syndrome sign dropped": ("int neg = s[c];", "int neg = 0;"),
    "message sign test inverted": ("if (x < 0.0f) neg ^= 1;", "if (x > 0.0f) neg ^= 1;"),
    "own edge kept in the check minimum": ("        if (e == own) continue;\n        float x", "        float x"),
    "own message kept in the exclusion sum": ("        if (k2 != k) a = a + mcv[k2];\n      msg[g->col_edge[b + k]] = store_msg",
                                              "        a = a + mcv[k2];\n      msg[g->col_edge[b + k]] = store_msg"),
    "scaling factor not applied": ("float mag = alpha * mn;", "float mag = mn;"),
    "posterior without the prior": ("    float L = lam[v];                       /* posterior */",
                                    "    float L = 0.0f;                         /* posterior */"),
    "schedule ignored": ("    int v = (int)perm[idx];\n    int b = g->colptr[v], deg = g->colptr[v + 1] - b;\n    for (int k = 0; k < deg; ++k) {         /* check",
                         "    int v = idx;\n    int b = g->colptr[v], deg = g->colptr[v + 1] - b;\n    for (int k = 0; k < deg; ++k) {         /* check"),
    "prior LLR transposed": ("log((1.0 - priors[j]) / priors[j])", "log(priors[j] / (1.0 - priors[j]))"),
    "heaviest candidate chosen": ("if (chosen < 0 || W < bestW) { bestW = W; chosen = i; }",
                                  "if (chosen < 0 || W > bestW) { bestW = W; chosen = i; }"),
    "average not normalised": ("(!isfinite(post[j]) ? post[j] : (nrm == 0.0f ? 0.0f : post[j] / nrm))",
                               "(!isfinite(post[j]) ? post[j] : post[j])"),
    "LSD grows along the worst column": ("if (w->col_root[j] < 0 && (best < 0 || ranks_before(soft, j, best))) best = j;",
                                         "if (w->col_root[j] < 0 && (best < 0 || ranks_before(soft, best, j))) best = j;"),
    "LSD right-hand side misread": ("int val = w->mat[pr * wd + ncol];", "int val = w->mat[pr * wd + 0];"),
    "LLR norm summed in one sequential pass": (
        "        for (int off = 16; off >= 1; off >>= 1) {\n"
        "          float nxt[32];\n"
        "          for (int l = 0; l < 32; ++l) nxt[l] = part[l] + part[l ^ off];\n"
        "          memcpy(part, nxt, sizeof(part));\n"
        "        }\n",
        "        { float seq = 0.0f;\n"
        "          for (int j = 0; j < n; ++j) seq = seq + (isfinite(post[j]) ? post[j] * post[j] : 0.0f);\n"
        "          part[0] = seq; }\n"),
    "correction limit off by one": ("if (nconv >= M) { t_stop = t; break; }", "if (nconv > M) { t_stop = t; break; }"),
}

PIN_SUITES = ["tests/test_oracle_bp.py", "tests/test_oracle_decoder.py", "tests/test_oracle_lsd.py"]

# mistakes in the parallel-schedule (flooding) member, run against its own pins
FLOOD_MUTATIONS = {
    "flooding posterior without the prior": ("    float L = lam[v];\n    for (int k = 0; k < deg; ++k) L = L + c2v[",
                                             "    float L = 0.0f;\n    for (int k = 0; k < deg; ++k) L = L + c2v["),
    "flooding own message kept in the exclusion sum": ("        if (k2 != k) a = a + c2v[g->col_edge[b + k2]];\n      msg[g->col_edge[b + k]] = store_msg",
                                                       "        a = a + c2v[g->col_edge[b + k2]];\n      msg[g->col_edge[b + k]] = store_msg"),
    "flooding uses messages of the same iteration": ("      c2v[own] = neg ? -mag : mag;\n    }\n  for (int v = 0; v < g->n; ++v) {          /* every posterior and variable-to-check message */\n    int b = g->colptr[v], deg = g->colptr[v + 1] - b;\n    float L",
                                                     "      c2v[own] = neg ? -mag : mag;\n      msg[own] = lam[g->edge_col[own]] + c2v[own];\n    }\n  for (int v = 0; v < g->n; ++v) {          /* every posterior and variable-to-check message */\n    int b = g->colptr[v], deg = g->colptr[v + 1] - b;\n    float L"),
    "flooding scaling factor not applied": ("      float mag = alpha * mn;\n      c2v[own]", "      float mag = mn;\n      c2v[own]"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) >= 1, f"mutation site not found: {name}"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "liboracle_mut.so"))
    env = dict(os.environ, VIBE_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PIN_SUITES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the planted mistake '{name}':\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", sorted(FLOOD_MUTATIONS))
def test_planted_flooding_mistake_is_caught(name, tmp_path):
    old, new = FLOOD_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) >= 1, f"mutation site not found: {name}"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "liboracle_mut.so"))
    env = dict(os.environ, VIBE_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_flood.py"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the planted mistake '{name}':\n{r.stdout[-2000:]}"


MEMBER_ALPHA_MUTATIONS = {
    "every member takes the first member's factor": ("prm->member_alpha ? prm->member_alpha[i] : prm->alpha",
                                                     "prm->member_alpha ? prm->member_alpha[0] : prm->alpha"),
    "member factors ignored": ("prm->member_alpha ? prm->member_alpha[i] : prm->alpha", "prm->alpha"),
}


@pytest.mark.parametrize("name", sorted(MEMBER_ALPHA_MUTATIONS))
def test_planted_member_alpha_mistake_is_caught(name, tmp_path):
    old, new = MEMBER_ALPHA_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site not found: {name}"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "liboracle_mut.so"))
    env = dict(os.environ, VIBE_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_decoder.py"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the planted mistake '{name}':\n{r.stdout[-2000:]}"


LAYERED_MUTATIONS = {
    "layers ignore shared variables": ("    while (taken[l]) ++l;\n", "    while (0) ++l;\n"),
    "layered check messages not kept between iterations": (
        "                        float* c2v, float* post) {\n  for (int l = 0; l < g->nlayer; ++l) {",
        "                        float* c2v, float* post) {\n  memset(c2v, 0, sizeof(float) * (size_t)g->E);\n"
        "  for (int l = 0; l < g->nlayer; ++l) {"),
    "layered update refreshes only the layer's own edge": (
        "        for (int k = 0; k < deg; ++k) {\n          float a = lam[v];",
        "        for (int k = 0; k < deg; ++k) {\n          if (g->col_edge[b + k] != ce) continue;\n"
        "          float a = lam[v];"),
    "layered posterior without the prior": ("    float L = lam[v];\n    for (int k = 0; k < deg; ++k) L = L + c2v[g->col_edge[b + k]];\n    post[v] = L;",
                                            "    float L = 0.0f;\n    for (int k = 0; k < deg; ++k) L = L + c2v[g->col_edge[b + k]];\n    post[v] = L;"),
}


@pytest.mark.parametrize("name", sorted(LAYERED_MUTATIONS))
def test_planted_layered_mistake_is_caught(name, tmp_path):
    old, new = LAYERED_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site not found: {name}"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "liboracle_mut.so"))
    env = dict(os.environ, VIBE_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_layered.py"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the planted mistake '{name}':\n{r.stdout[-2000:]}"


LSD_ORDER_MUTATIONS = {
    "order search one column short": ("      int qn = order < nfree ? order : nfree;",
                                      "      int qn = order < nfree ? order - 1 : nfree;"),
    "order search keeps the heaviest setting": ("        if (a == 0 || W < bestW) { bestW = W;",
                                                "        if (a == 0 || W > bestW) { bestW = W;"),
    "order search over the last free columns": (
        "        for (int b = 0; b < qn; ++b) w->x[w->tmp[b]] = (uint8_t)((a >> b) & 1);\n"
        "        for (int t = 0; t < ncol; ++t) {\n"
        "          int pr = w->pivrow[t];\n"
        "          if (pr < 0) continue;\n"
        "          int val = w->mat[pr * wd + ncol];\n"
        "          for (int b = 0; b < qn; ++b) val ^= w->mat[pr * wd + w->tmp[b]] & w->x[w->tmp[b]];",
        "        for (int b = 0; b < qn; ++b) w->x[w->tmp[nfree - 1 - b]] = (uint8_t)((a >> b) & 1);\n"
        "        for (int t = 0; t < ncol; ++t) {\n"
        "          int pr = w->pivrow[t];\n"
        "          if (pr < 0) continue;\n"
        "          int val = w->mat[pr * wd + ncol];\n"
        "          for (int b = 0; b < qn; ++b) val ^= w->mat[pr * wd + w->tmp[nfree - 1 - b]] & w->x[w->tmp[nfree - 1 - b]];"),
}


@pytest.mark.parametrize("name", sorted(LSD_ORDER_MUTATIONS))
def test_planted_lsd_order_mistake_is_caught(name, tmp_path):
    old, new = LSD_ORDER_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site not found: {name}"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "liboracle_mut.so"))
    env = dict(os.environ, VIBE_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_lsd.py"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the planted mistake '{name}':\n{r.stdout[-2000:]}"
