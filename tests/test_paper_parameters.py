"""The workload's parameters are the ones the paper prints for its runs
(tests/golden/paper_parameters.txt, Sec. 2)."""
import inspect
import os

import numpy as np

from paper_0911_2889_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _golden():
    vals = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_parameters.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            name, value = line.split()[:2]
            vals[name] = float(value)
    return vals


def test_bench_workload_uses_the_paper_parameters():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    g = _golden()
    assert bench.WORKLOAD["gamma"] == g["gamma"]
    assert bench.WORKLOAD["t0"] == g["t0"]


def test_initial_conditions_use_the_paper_amplitude():
    g = _golden()
    assert inspect.signature(inputs.physical_ic).parameters["eps"].default == g["eps"]
    assert inspect.signature(inputs.spectrum_ic).parameters["amp"].default == g["eps"]
    field = inputs.physical_ic(32, 64, seed=0)
    assert np.abs(field).max() <= g["eps"]


def test_the_step_has_no_forcing():
    # with f = 0 and a zero state, nothing moves: Phi stays 0, the mean mode
    # stays 0 (the oracle's step is the reference for the GPU path)
    from oracle import oracle as orc
    g = _golden()
    assert g["forcing"] == 0
    p = orc.Params(n1=16, n2=32, K1=3, K2=7, gamma=g["gamma"], s1=1.0, s2=1.0, t0=g["t0"], dt=1e-3)
    s, m, t = orc.step(p, np.zeros(p.box_shape, dtype=np.complex128), 0.0, g["t0"], 5)
    assert not np.any(s) and m == 0.0 and t == g["t0"] + 5e-3
