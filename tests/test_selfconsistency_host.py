"""Host logic of the self-consistency loop of Sec. IV.C (paper_1309_5994_gb300.selfconsistency)
with a stand-in solver on CPU: the stopping rule on the paper's measure, the reuse of the
local-Green's-function buffer between iterations, and the mixing options passed through."""
from types import SimpleNamespace

from paper_1309_5994_gb300.selfconsistency import self_consistent


class _LoopFake:
    def __init__(self, measures):
        self.measures = list(measures)
        self.outs, self.steps, self.depth = [], [], None

    def set_anderson(self, depth):
        self.depth = depth

    def local_greens(self, sources, precision=0, tol=0.0, max_sweeps=0, out=None):
        assert sources is None                            # every site
        out = object() if out is None else out
        self.outs.append(out)
        return out, SimpleNamespace(report={"sweeps": 3})

    def selfenergy_step(self, gloc, mix):
        assert gloc is self.outs[-1]                      # the step sees this iteration's G_loc
        self.steps.append(mix)
        return self.measures.pop(0)


def test_loop_stops_at_the_measure_and_reuses_its_buffer():
    s = _LoopFake([1e-2, 1e-5, 5e-9, 1e-12])
    r = self_consistent(s, mix=0.6, anderson=3)
    assert r["converged"] and r["iterations"] == 3 and r["delta_sc"] == 1e-8
    assert r["history"] == [1e-2, 1e-5, 5e-9]
    assert len({id(o) for o in s.outs}) == 1 and s.steps == [0.6] * 3 and s.depth == 3
    assert [q["sweeps"] for q in r["reports"]] == [3, 3, 3]


def test_loop_reports_no_convergence_at_max_iter():
    s = _LoopFake([1.0, 0.5, 0.25, 0.125])
    r = self_consistent(s, delta_sc=1e-3, max_iter=3)
    assert not r["converged"] and r["iterations"] == 3 and r["history"] == [1.0, 0.5, 0.25]
    assert s.depth == 0                                   # linear mixing unless asked otherwise
