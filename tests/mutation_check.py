"""Mutation check of the oracle's pins (CPU only; not collected by pytest).

Each entry plants one plausible mistake (a dropped term, a wrong sign,
index or comparison) in a temporary copy of the oracle sources, builds that
copy, and runs the oracle pins (tests/test_oracle_*.py) against it through
KPO_LIB.  A pin set that lets a planted mistake pass has a hole.  The
oracle in the tree is never modified.

    python tests/mutation_check.py [substring of a mutation's name]

Exit status 0 when every planted mistake fails at least one pin.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle.build import compile_oracle  # noqa: E402

# (file, original text, planted text, what it breaks)
MUTATIONS = [
    # Eq. 3-5 (Algorithm 3)
    ("planner.c", "double freevol = ((delta + nv) * vol) / ((delta + nv) + ni);",
     "double freevol = (nv * vol) / ((delta + nv) + ni);", "Eq. 3: delta dropped from the numerator"),
    ("planner.c", "double den = (1.0 + (double)cov[i]) * (1.0 + n_all * n_all);",
     "double den = (1.0 + (double)cov[i]) * (1.0 + nv * nv);", "Eq. 4: invalid samples dropped"),
    ("planner.c", "double f4 = (freevol * freevol) * (freevol * freevol);",
     "double f4 = (freevol * freevol) * freevol;", "Eq. 4: cube instead of fourth power"),
    ("planner.c", "p = score[i] / sum + eps;", "p = score[i] / sum;", "Eq. 5: eps dropped"),
    ("planner.c", "    if (!avail[i]) continue;\n", "", "Eq. 3-4: scores outside R_avail"),
    # Algorithm 2: representatives and the accept draw
    ("planner.c", "  for (int key = 0; key < S; ++key) {\n    if ((fl[key] & 2) && !claimed[ss[key]]) {",
     "  for (int key = S - 1; key >= 0; --key) {\n    if ((fl[key] & 2) && !claimed[ss[key]]) {",
     "Algorithm 2: largest key represents a sub-region"),
    ("planner.c", "if ((uint64_t)w1[1] < o->thr[r]) f |= 4;", "if ((uint64_t)w1[0] < o->thr[r]) f |= 4;",
     "Algorithm 2: accept draw from the duration word"),
    # Eq. 6 and Algorithm 4
    ("planner.c", "int32_t lam = room / n_ve; /* floor: both non-negative */",
     "int32_t lam = (room + n_ve - 1) / n_ve;", "Eq. 6: ceiling instead of floor"),
    ("planner.c", "    o->in_ve[id] = 1;", "    o->in_ve[id] = 0;", "Algorithm 4: new nodes left out of V_E"),
    ("planner.c", "o->in_ve[v] = (uint64_t)w[0] < o->thr[o->region[v]] ? 1 : 0;",
     "o->in_ve[v] = (uint64_t)w[1] < o->thr[o->region[v]] ? 1 : 0;", "Algorithm 4: wrong draw word"),
    # validity (Sec. II valid set) and binning (Sec. III)
    ("model.c", "    if (sep <= 0.0) {", "    if (sep < 0.0) {", "obstacles as open sets"),
    ("model.c", "if (!(lo <= x[i] && x[i] <= hi)) {", "if (!(lo < x[i] && x[i] <= hi)) {",
     "state box open at its lower bound"),
    ("model.c", "  else if (t >= (double)n)\n    i = n - 1;", "  else if (t > (double)n)\n    i = n - 1;",
     "binning: top clamp off by one"),
    ("model.c", "    double t = speed_of(o, x) * ((double)o->cfg.speed_bins / o->cfg.speed_hi);",
     "    double t = speed_of(o, x) * speed_of(o, x) * ((double)o->cfg.speed_bins / o->cfg.speed_hi);",
     "binning: squared speed in the speed bins"),
    ("model.c", "      const double y = x[dd] - 2.0 * pi * floor((x[dd] + pi) / (2.0 * pi));\n      t = (y + pi) * ((double)n / (2.0 * pi));",
     "      const double y = x[dd] - 2.0 * pi * floor(x[dd] / (2.0 * pi));\n      t = y * ((double)n / (2.0 * pi));",
     "binning: angle wrapped to [0, 2 pi)"),
    ("model.c", "  int r = cell[0] + gx * (cell[1] + gy * (cell[2] + gz * (sb + nsb * e)));",
     "  int r = cell[2] + gz * (cell[1] + gy * (cell[0] + gx * (sb + nsb * e)));",
     "binning: region index with x slowest"),
    # learned proposal features (reading R13)
    ("planner.c", "for (int a = 0; a < 3; ++a) f[6 + a] = o->cfg.goal_c[a] - x[a];",
     "for (int a = 0; a < 3; ++a) f[6 + a] = x[a] - o->cfg.goal_c[a];",
     "features: goal offset with the wrong sign"),
    # free-space-obeying decomposition (Sec. IV-B, kd-tree over obstacle faces)
    ("model.c", "      split = cand[(u - 1) / 2];", "      split = cand[u / 2];",
     "kd-tree: upper instead of lower median"),
    ("model.c", "    if (u > best_m) {", "    if (u > 0 && u >= best_m) {",
     "kd-tree: ties to the highest axis"),
    # Dubins airplane field
    ("model.c", "  dx[0] = v * cos(psi) * cos(theta);", "  dx[0] = v * cos(psi) * sin(theta);",
     "Dubins: x rate with sin(theta)"),
    ("model.c", "  dx[4] = u[1];", "  dx[4] = u[2];", "Dubins: pitch rate from the wrong control"),
    # Philox4x32-10 (Salmon et al., SC'11)
    ("philox.c", "    if (round > 0) { /* key schedule", "    if (round > 1) { /* key schedule",
     "Philox: key bumped one round late"),
    ("philox.c", "    uint32_t y0 = hi1 ^ x1 ^ k0;", "    uint32_t y0 = hi1 ^ x3 ^ k0;",
     "Philox: wrong word mixed into y0"),
    # learned proposal network and Adam
    ("mlp.c", "draw[i] = -z * exp(-ls) * (1.0 - mu * mu) / (double)M;",
     "draw[i] = -z * exp(-ls) / (double)M;", "MLP: tanh derivative dropped"),
    ("mlp.c", "s += dh2[n] * q.W2[n * H + k];", "s += dh2[n] * q.W2[k * H + n];",
     "MLP: backward through W2 untransposed"),
    ("mlp.c", "const double mh = m[i] / c1, vh = v[i] / c2;", "const double mh = m[i] / c1, vh = v[i];",
     "Adam: second-moment bias correction dropped"),
    # quadrotor field
    ("model.c", "double bz_x = cphi * stheta * cpsi + sphi * spsi;",
     "double bz_x = cphi * stheta * cpsi - sphi * spsi;", "quadrotor: thrust direction sign (x)"),
    ("model.c", "double bz_y = cphi * stheta * spsi - sphi * cpsi;",
     "double bz_y = cphi * stheta * spsi + sphi * cpsi;", "quadrotor: thrust direction sign (y)"),
    ("model.c", "dx[4] = cphi * q - sphi * r;", "dx[4] = cphi * q + sphi * r;",
     "quadrotor: Euler-rate map sign"),
    ("model.c", "dx[3] = p + sphi * ttheta * q + cphi * ttheta * r;",
     "dx[3] = p + cphi * ttheta * q + sphi * ttheta * r;", "quadrotor: Euler-rate map entries swapped"),
    ("model.c", "double gx = q * Lz - r * Ly;", "double gx = r * Ly - q * Lz;",
     "quadrotor: gyroscopic term sign"),
    ("model.c", "double tau_x = l * (T2 - T4);", "double tau_x = l * (T3 - T1);",
     "quadrotor: roll torque from the pitch rotors"),
    # the work count behind the roofline (oracle/work.c)
    ("work.c", "  o->work.steps += 1;", "  o->work.steps += 2;", "work: every step counted twice"),
    ("work.c", "    if (!(lo <= x1[i] && x1[i] <= hi)) return; /* no hull test */\n", "",
     "work: a hull counted for a step that left the state box"),
    ("work.c", "  o->work.samples += 1;", "  o->work.samples += 1 + (o->work.samples == 0);",
     "work: one sample too many"),
]


def run_pins(lib: str) -> int:
    env = dict(os.environ, KPO_LIB=lib)
    tests = sorted(glob.glob(os.path.join(ROOT, "tests", "test_oracle_*.py")))
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                            *tests], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        return r.returncode
    except subprocess.TimeoutExpired:
        return -1


def main() -> int:
    sel = sys.argv[1] if len(sys.argv) > 1 else ""
    src = os.path.join(ROOT, "oracle")
    survivors = []
    with tempfile.TemporaryDirectory() as tmp:
        for f in os.listdir(src):
            if f.endswith((".c", ".h")):
                shutil.copy(os.path.join(src, f), tmp)
        lib = os.path.join(tmp, "libkpo_base.so")
        compile_oracle(tmp, lib)
        if run_pins(lib) != 0:
            print("the unmodified oracle fails its pins")
            return 2
        for fname, old, new, what in MUTATIONS:
            if sel not in what:
                continue
            path = os.path.join(tmp, fname)
            orig = open(path).read()
            if orig.count(old) != 1:
                print(f"{what}: text to mutate not found once")
                return 2
            with open(path, "w") as f:
                f.write(orig.replace(old, new))
            lib = os.path.join(tmp, "libkpo_mut.so")
            compile_oracle(tmp, lib)
            rc = run_pins(lib)
            with open(path, "w") as f:
                f.write(orig)
            caught = rc != 0
            print(f"{'caught ' if caught else 'MISSED '} {what}", flush=True)
            if not caught:
                survivors.append(what)
    print(f"{len(survivors)} planted mistakes passed the pins")
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main())
