"""The rule of the DGAL_VALIDATE input check (every vertex strictly left of
every edge it is not an end of) is strict convexity in counter-clockwise
order: pinned against an independent form, the polygon being its own strict
convex hull in the hull's counter-clockwise order (Andrew's monotone chain),
in exact rational arithmetic."""
from collections import Counter

from .validate_rule import families, is_own_strict_hull, passes


def test_rule_equals_own_strict_hull():
    P, C, names = families(n=150)
    outcome = Counter()
    for p, m, name in zip(P, C, names):
        a = passes(p, int(m))
        assert a == is_own_strict_hull(p, int(m)), (name, p[: int(m)].tolist())
        outcome[(name, a)] += 1
    for name in ("hull", "quad", "square"):
        assert outcome[(name, False)] == 0, name
    for name in ("clockwise", "bowtie", "reflex", "repeated", "collinear", "pentagram"):
        assert outcome[(name, True)] == 0, name
    # vertices a few ulps off the line of their neighbours fall on both sides
    assert outcome[("nudged", True)] > 10 and outcome[("nudged", False)] > 10
