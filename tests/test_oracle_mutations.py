"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of the oracle's C source (a changed
constant, sign, word, range, neighbour or index), compiles it and runs the
pin tests (test_oracle_pins.py) against that copy in a child process: at
least one pin must fail.  The unchanged source, compiled the same way, must
pass them all, so a failure is the planted mistake's and not the harness's.
The same is done for the Python oracles of the finite-size-scaling,
multi-histogram and ladder rows: the child process replaces the oracle
submodule with the changed copy before running that row's pin tests.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "xy_oracle.c")

# name -> (original text, planted text); each original occurs once.
MUTATIONS = {
    "Philox multiplier": ("const uint32_t M0 = 0xD2511F53u", "const uint32_t M0 = 0xD2511F55u"),
    "Philox round count": ("for (int round = 0; round < 10; ++round)", "for (int round = 0; round < 9; ++round)"),
    "odd site takes the words swapped": ("*wa = w[2];\n    *wb = w[3];", "*wa = w[3];\n    *wb = w[2];"),
    "initial angles over half the circle": ("th[site(Lx, Ly, x, y, z)] = XO_TWO_PI * xo_u01(wa);",
                                            "th[site(Lx, Ly, x, y, z)] = 0.5 * XO_TWO_PI * xo_u01(wa);"),
    "initial angle from the acceptance word": ("th[site(Lx, Ly, x, y, z)] = XO_TWO_PI * xo_u01(wa);",
                                               "th[site(Lx, Ly, x, y, z)] = XO_TWO_PI * xo_u01(wb);"),
    "energy change with the wrong sign": ("double dE = -(hx * (cos(t_new) - cos(t_old)) +",
                                          "double dE = (hx * (cos(t_new) - cos(t_old)) +"),
    "acceptance without beta": ("double a = exp(-beta * dE);", "double a = exp(-dE);"),
    "over-relaxation leaves the spin": ("if (t >= XO_TWO_PI) t = 0.0;\n        th[i] = t;",
                                        "if (t >= XO_TWO_PI) t = 0.0;\n        (void)t;"),
    "reflection with the wrong sign": ("double Spx = -Sx + 2.0 * d / H2 * Hx;", "double Spx = Sx + 2.0 * d / H2 * Hx;"),
    "only one neighbour per axis": ("for (int sgn = -1; sgn <= 1; sgn += 2) {", "for (int sgn = 1; sgn <= 1; sgn += 2) {"),
    "exchange exponent with the wrong sign": ("double expo = (betas[k] - betas[k + 1]) * (E[rm] - E[rn]);",
                                              "double expo = (betas[k + 1] - betas[k]) * (E[rm] - E[rn]);"),
    "helicity sine with the wrong orientation": ("S[mu] += sin(ti - tj);", "S[mu] += sin(tj - ti);"),
    "bond counted twice": ("C[mu] += cos(ti - tj);", "C[mu] += 2.0 * cos(ti - tj);"),
    "reweighting weight with the wrong sign": ("double w = exp(-db * E[t] - lz);", "double w = exp(db * E[t] - lz);"),
    "covariance with the wrong sign": ("cov[(long)k * n_obs + j] = sOE[j] - sO[j] * sE;",
                                       "cov[(long)k * n_obs + j] = sO[j] * sE - sOE[j];"),
}


def _pins_pass(src_text, workdir):
    """Compile the given oracle source and run the pin tests against it;
    True if every pin passed."""
    os.makedirs(workdir, exist_ok=True)
    c_path, so_path = os.path.join(workdir, "xy_oracle.c"), os.path.join(workdir, "liboracle.so")
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99", "-o", so_path, c_path, "-lm"],
                   check=True)
    env = dict(os.environ, XY_ORACLE_LIBRARY=so_path, OMP_NUM_THREADS="1")
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return res.returncode == 0


def test_every_planted_mistake_fails_a_pin(tmp_path):
    with open(SRC) as f:
        src = f.read()
    jobs = {"unchanged": src}
    for name, (orig, planted) in MUTATIONS.items():
        assert src.count(orig) == 1, name
        jobs[name] = src.replace(orig, planted)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futures = {name: ex.submit(_pins_pass, text, str(tmp_path / f"m{i}"))
                   for i, (name, text) in enumerate(jobs.items())}
        passed = {name: fut.result() for name, fut in futures.items()}
    assert passed["unchanged"], "the unchanged oracle must pass its pins"
    survivors = [name for name in MUTATIONS if passed[name]]
    assert not survivors, f"planted mistakes no pin caught: {survivors}"


# Python oracle submodule -> [(name, original text, planted text)]
PY_MUTATIONS = {
    "fss": [
        ("each bin loses its last sample", "np.tile(np.arange(edges[b], edges[b + 1]), int(n))",
         "np.tile(np.arange(edges[b], edges[b + 1] - 1), int(n))"),
        ("1/nu from the inverted slope ratio", "inv_nu = np.log(abs(sB) / abs(sA)) / np.log(LB / LA)",
         "inv_nu = np.log(abs(sA) / abs(sB)) / np.log(LB / LA)"),
        ("slopes of the swapped curves", "sA, sB = dfA(root), dfB(root)", "sA, sB = dfB(root), dfA(root)"),
    ],
    "multihist": [
        ("record counts left out", "a = np.log(np.asarray(counts, np.float64))[None, :] + np.asarray(f)[None, :] \\",
         "a = 0.0 * np.log(np.asarray(counts, np.float64))[None, :] + np.asarray(f)[None, :] \\"),
        ("free energies with the wrong sign", "+ np.asarray(f)[None, :] \\", "- np.asarray(f)[None, :] \\"),
        ("covariance with the wrong sign", "out_cov.append(w @ (O * E[:, None]) - mO * mE)",
         "out_cov.append(mO * mE - w @ (O * E[:, None]))"),
        ("normalised at the last coupling", "fn -= fn[0]", "fn -= fn[-1]"),
    ],
    "ladder": [
        ("widths along sigma instead of 1/sigma", "target = (1.0 / sigma) / np.sum(1.0 / sigma) * (b[-1] - b[0])",
         "target = sigma / np.sum(sigma) * (b[-1] - b[0])"),
        ("damping the wrong way", "new_width = (1.0 - damping) * width + damping * target",
         "new_width = damping * width + (1.0 - damping) * target"),
    ],
}
PY_PINS = {"fss": "test_fss_oracle.py", "multihist": "test_multihist_oracle.py", "ladder": "test_ladder.py"}

BOOT = r"""
import sys, types
sys.path.insert(0, sys.argv[1])
import oracle
name, path, tests = sys.argv[2], sys.argv[3], sys.argv[4]
m = types.ModuleType("oracle." + name)
m.__package__ = "oracle"
m.__file__ = path
exec(compile(open(path).read(), path, "exec"), m.__dict__)
sys.modules["oracle." + name] = m
setattr(oracle, name, m)
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", tests]))
"""


def _py_pins_pass(module, src_text, workdir):
    os.makedirs(workdir, exist_ok=True)
    path = os.path.join(workdir, module + ".py")
    with open(path, "w") as f:
        f.write(src_text)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run([sys.executable, "-c", BOOT, ROOT, module, path, os.path.join(ROOT, "tests", PY_PINS[module])],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return res.returncode == 0


def test_every_planted_mistake_in_the_python_oracles_fails_a_pin(tmp_path):
    jobs = {}
    for module, muts in PY_MUTATIONS.items():
        with open(os.path.join(ROOT, "oracle", module + ".py")) as f:
            src = f.read()
        jobs[(module, "unchanged")] = (module, src)
        for name, orig, planted in muts:
            assert src.count(orig) == 1, name
            jobs[(module, name)] = (module, src.replace(orig, planted))
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futures = {key: ex.submit(_py_pins_pass, mod, text, str(tmp_path / f"p{i}"))
                   for i, (key, (mod, text)) in enumerate(jobs.items())}
        passed = {key: fut.result() for key, fut in futures.items()}
    assert all(passed[(m, "unchanged")] for m in PY_MUTATIONS), passed
    survivors = [key for key, ok in passed.items() if key[1] != "unchanged" and ok]
    assert not survivors, f"planted mistakes no pin caught: {survivors}"
