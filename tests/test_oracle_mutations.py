"""Planted mistakes in a copy of the oracle must make the pins fail.

Each mutation is a plausible slip (a flipped sign, a dropped term, a wrong
index, a transposed operand, a wrong comparison).  The test compiles a
mutated copy of oracle/dgal_oracle.c into a temporary library, runs the pin
suite against it in a child process and expects a failure.  The shipped
oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dgal_oracle.c")

MUTATIONS = [
    ("orient operands transposed", "return cross2(sub2(b, a), sub2(p, a));", "return cross2(sub2(p, a), sub2(b, a));"),
    ("crossing t operands transposed", "*t = cross2(q, s) / *D;", "*t = cross2(s, q) / *D;"),
    ("crossing strictness lost", "return (*t > 0.0 && *t < 1.0", "return (*t >= 0.0 && *t <= 1.0"),
    ("duplicate-vertex rule dropped", "if (!dup && inside_or_on(Q[j], P, n1))", "if (inside_or_on(Q[j], P, n1))"),
    ("rotation to largest code", "if (cand[k].code < cand[s0].code) s0 = k;", "if (cand[k].code > cand[s0].code) s0 = k;"),
    ("union without -A_i", "double U = out->a1 + out->a2 - out->ai;", "double U = out->a1 + out->a2;"),
    ("shoelace adjoint term dropped", "opt gw = {0.5 * gai * (wn.y - wp.y), 0.5 * gai * (wp.x - wn.x)};",
     "opt gw = {0.5 * gai * (wn.y), 0.5 * gai * (wp.x - wn.x)};"),
    ("dD sign flipped", "double gN = gt / D, gD = -gt * t / D;", "double gN = gt / D, gD = gt * t / D;"),
    ("crossing grad to wrong vertex", "g1[i1].x += gr.x;", "g1[i].x += gr.x;"),
    ("area-gradient sign flipped", "double ga12 = -g * ai / (U * U);", "double ga12 = g * ai / (U * U);"),
    ("gs term dropped", "opt gs = {gN * (-q.y) + gD * (-r.y), gN * q.x + gD * r.x};",
     "opt gs = {gN * (-q.y), gN * q.x + gD * r.x};"),
    ("P2 gradient index shifted", "g2[j1].x += gs.x;", "g2[j].x += gs.x;"),
    # the near-degenerate classifier, which decides where bit-exactness is waived
    ("orientation threshold x10", "double thr = ORC_DEGEN_REL * L * L;", "double thr = 10.0 * ORC_DEGEN_REL * L * L;"),
    ("crossing-parameter threshold x10", "if (t <= ORC_DEGEN_REL || t >= 1.0 - ORC_DEGEN_REL) return 1;",
     "if (t <= 10.0 * ORC_DEGEN_REL || t >= 1.0 - 10.0 * ORC_DEGEN_REL) return 1;"),
    ("parallel-edge threshold x10", "if (fabs(cross2(r, s)) <= ORC_DEGEN_REL * nr * ns && bbox_overlap",
     "if (fabs(cross2(r, s)) <= 10.0 * ORC_DEGEN_REL * nr * ns && bbox_overlap"),
    ("parallel-edge bbox guard dropped", "ORC_DEGEN_REL * nr * ns && bbox_overlap(a, b, c, d)) return 1;",
     "ORC_DEGEN_REL * nr * ns) return 1;"),
    ("classifier scale L about the origin", "opt o = P[0];", "opt o = {0.0, 0.0};"),
    # the GIoU / DIoU loss terms
    ("hull keeps right turns", "while (h >= 2 && orient(hull[h - 2].p, hull[h - 1].p, pts[k].p) <= 0.0) --h;",
     "while (h >= 2 && orient(hull[h - 2].p, hull[h - 1].p, pts[k].p) >= 0.0) --h;"),
    ("GIoU hull-area gradient sign", "double gh = w * U / (hq.ah * hq.ah);", "double gh = -w * U / (hq.ah * hq.ah);"),
    ("GIoU 1 / A_h term dropped from dL/dA_i", "gai = w * (-di + 1.0 / hq.ah);", "gai = w * (-di);"),
    ("DIoU centre gradient to the wrong polygon",
     "g2[j].x -= gr * 2.0 * (m1.x - m2.x) / n2;", "g2[j].x += gr * 2.0 * (m1.x - m2.x) / n2;"),
    ("DIoU diameter from the wrong pair", "if (d > o->c2) { o->c2 = d; o->da = a; o->db = b; }",
     "if (d > o->c2) { o->c2 = d; o->da = a; o->db = a; }"),
    ("DIoU centre as the first vertex", "m1.x /= n1; m1.y /= n1; m2.x /= n2; m2.y /= n2;\n    o->rho2",
     "m1 = P[0]; m2 = Q[0];\n    o->rho2"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(tmp_path, name, old, new):
    src = open(SRC).read()
    old, new = old.replace("\\n", "\n"), new.replace("\\n", "\n")
    assert src.count(old) == 1, f"mutation anchor not found: {name}"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(mut), "-lm"],
                   check=True)
    env = dict(os.environ, DGAL_ORACLE_SO=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_loss_variants.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
