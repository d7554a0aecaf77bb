"""Planted mistakes in a copy of the oracle are caught by pins that do not use
the oracle.

Each case copies oracle/ to a temporary directory, changes one line of the
copied pamc.c into a plausible mistake, builds that copy and runs pins
computed independently of the oracle:
  * <E> and beta F_k = -ln Z(beta_k) of the anneal against numpy enumeration
    of the 4 x 4 torus (+-J without field; Gaussian couplings with a field),
    z-tests over eight seeds (Sec. II.A, Eq. 1; Sec. II.B);
  * the energies the run reports against a numpy recompute from its spins;
  * multinomial resampling on fixed energies: copy numbers against numpy
    weights (chi-square) and ln Q against its numpy value.
The unmodified oracle passes the same pins; every mutant fails at least one.
The committed oracle is never modified.
"""
import importlib.util
import math
import shutil

import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W

PM1, REAL = 0, 1
D, L, N = 2, 4, 16
BETAS = W.schedule_lb(11, 1.5)
KS = (5, 10)

# (description, file, original line fragment, planted line fragment)
MUTANTS = [
    ("field sign in the local field", "pamc.c",
     "f = f + (c->h ? c->h[i] : 0.0f);", "f = f - (c->h ? c->h[i] : 0.0f);"),
    ("neighbour sign in the local field", "pamc.c",
     "float t = sr[c->nbr[i * twoD + nb]] > 0 ? Jb : -Jb;", "float t = sr[c->nbr[i * twoD + nb]] > 0 ? -Jb : Jb;"),
    ("threshold of the wrong energy change", "pamc.c",
     "thr[n] = or_threshold_pm(beta, 4 * n);", "thr[n] = or_threshold_pm(beta, 2 * n);"),
    ("energy change off by one class", "pamc.c",
     "int dE = 4 * c->D - 4 * n_unsat;", "int dE = 4 * c->D - 4 * n_unsat - 4;"),
    ("periodic wrap", "pamc.c",
     "cp = (c + 1) % L;", "cp = (c + 1) % (L - 1);"),
    ("field sign in the energy", "pamc.c",
     "e -= (sr[i] > 0) ? fix96(c->h[i]) : -fix96(c->h[i]);", "e += (sr[i] > 0) ? fix96(c->h[i]) : -fix96(c->h[i]);"),
    ("weights with beta instead of the beta step", "pamc.c",
     "double db = beta_next - beta_prev;", "double db = beta_next;"),
    ("ln Q without the -ln R term", "pamc.c",
     "*lnQ = (-(db * e_to_double(kind, emin)) + log(S)) - log((double)R);",
     "*lnQ = (-(db * e_to_double(kind, emin)) + log(S));"),
    ("beta F sign", "pamc.c",
     "o[4] = -(double)s->N * log(2.0) - s->sum_lnQ;", "o[4] = -(double)s->N * log(2.0) + s->sum_lnQ;"),
    ("draw lands on the next replica", "pamc.c",
     "counts[lo] += 1;", "counts[lo + 1 < R ? lo + 1 : lo] += 1;"),
    ("weight exponent sign", "pamc.c",
     "w[r] = or_spec_exp64(-(db * e_to_double(kind, E[r] - emin)));",
     "w[r] = or_spec_exp64(-(db * e_to_double(kind, emin - E[r])));"),
]


def _states():
    idx = np.arange(1 << N, dtype=np.int64)
    return (1 - 2 * ((idx[:, None] >> np.arange(N)) & 1)).astype(np.float64)  # [state, site]


def _nbr_plus():
    # site i = x + L y; neighbour in +x and +y, periodic
    x, y = np.arange(N) % L, np.arange(N) // L
    return [((x + 1) % L) + L * y, x + L * ((y + 1) % L)]


def _energies(J, h, s):
    """E = -sum_{i,d} J[d N + i] s_i s_{i+e_d} - sum_i h_i s_i for spins s [.., N]."""
    J = np.asarray(J, np.float64)
    e = np.zeros(s.shape[:-1])
    for d, nb in enumerate(_nbr_plus()):
        e -= (J[d * N:(d + 1) * N] * s * s[..., nb]).sum(axis=-1)
    if h is not None:
        e -= (np.asarray(h, np.float64) * s).sum(axis=-1)
    return e


def _exact(J, h):
    E = _energies(J, h, _states())
    out = []
    for b in BETAS:
        a = -b * E
        m = a.max()
        w = np.exp(a - m)
        out.append((m + math.log(w.sum()), float((w * E).sum() / w.sum())))
    return out


def _load(path):
    spec = importlib.util.spec_from_file_location(f"oracle_copy_{abs(hash(str(path)))}", str(path / "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


def _failed_resampling_pins(O):
    """Multinomial resampling on fixed energies (Sec. II.B): copy numbers sum
    to R, their means follow R w_i / S with w_i from numpy (chi-square over
    100 draws of the population), and ln Q = -dbeta E_min + ln S - ln R."""
    fails = []
    rng = np.random.default_rng(42)
    R = 400
    E = rng.integers(-40, 0, R) * 4
    pairs = np.stack([E, -np.ones(R, np.int64)], 1).reshape(-1)
    w = np.exp(-0.05 * (E - E.min()))
    tot = np.zeros(R)
    M = 100
    for k in range(1, M + 1):
        r = O.resample(PM1, pairs, 1.0, 1.05, k, seed=9)
        if r["counts"].sum() != R:
            return ["resampling: population"]
        tot += r["counts"]
    expct = M * R * w / w.sum()
    chi2 = ((tot - expct) ** 2 / expct).sum()
    if not abs(chi2 - (R - 1)) < 6 * math.sqrt(2 * (R - 1)):
        fails.append("resampling: copy numbers")
    lnQ = -0.05 * E.min() + math.log(w.sum()) - math.log(R)
    if not abs(r["lnQ"] - lnQ) < 1e-10 * abs(lnQ):
        fails.append("resampling: ln Q")
    return fails


def _failed_pins(O):
    fails = _failed_resampling_pins(O)
    cases = [("pm", PM1, W.couplings_pm(D, L, 61).astype(np.float32), None),
             ("gauss+h", REAL, W.couplings_gauss(D, L, 62), W.field_uniform(N, 63))]
    for name, kind, J, h in cases:
        ex = _exact(J, h)
        E = {k: [] for k in KS}
        bF = {k: [] for k in KS}
        for seed in range(7000, 7008):
            s = O.Sim(D, L, kind, J, h, 800, BETAS, 6, seed)
            s.run()
            for k in KS:
                o = s.obs(k)
                E[k].append(o["E_mean"])
                bF[k].append(o["betaF"])
        # energies reported by the last run against a recompute from its spins
        spins = s.spins().astype(np.float64)
        got = np.array([float(e) for e in s.energies()])
        if kind == REAL:
            got = got * 2.0 ** -96
        if not np.allclose(got, _energies(J, h, spins), rtol=0, atol=1e-9):
            fails.append(f"{name}: energies")
        for k in KS:
            for what, vals, target in (("E", E[k], ex[k][1]), ("betaF", bF[k], -ex[k][0])):
                v = np.asarray(vals)
                se = max(v.std(ddof=1) / math.sqrt(len(v)), 1e-9)
                if not abs(v.mean() - target) < 5 * se:
                    fails.append(f"{name}: {what}[{k}]")
    return fails


@pytest.fixture(scope="module")
def oracle_src():
    import os
    return os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def test_unmodified_oracle_passes_the_pins(tmp_path, oracle_src):
    shutil.copytree(oracle_src, tmp_path / "oracle", ignore=shutil.ignore_patterns("_build", "__pycache__"))
    assert _failed_pins(_load(tmp_path / "oracle")) == []


@pytest.mark.parametrize("desc,fname,orig,planted", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, oracle_src, desc, fname, orig, planted):
    dst = tmp_path / "oracle"
    shutil.copytree(oracle_src, dst, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    src = (dst / fname).read_text()
    assert orig in src, desc
    (dst / fname).write_text(src.replace(orig, planted, 1))
    fails = _failed_pins(_load(dst))
    assert fails, f"planted mistake not caught: {desc}"
