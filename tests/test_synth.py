"""The seeded input recipe (paper_1205_0359_gb300/synth.py): properties its
workloads must have for the solver tests to mean what they claim."""
import numpy as np

from paper_1205_0359_gb300 import synth


def test_links_are_su3():
    rng = np.random.Generator(np.random.PCG64(3))
    U = synth.su3_links((2, 2, 4, 2), 0.6, rng).reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - eye).max() < 1e-12
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-12


def test_rhs_kinds_and_dependencies():
    z2 = synth.z2_rhs(1000, 2, np.random.Generator(np.random.PCG64(1)))
    assert np.allclose(np.abs(z2.real) * np.sqrt(2), 1.0) and np.allclose(np.abs(z2.imag) * np.sqrt(2), 1.0)
    w1 = synth.make_workload("w1_4x4x4x4")
    B = w1["B"]
    assert np.array_equal(B[3], B[0] + B[1])                      # exact dependence: deflation must trigger
    w5 = synth.make_workload("w5_32x32x32x64", dims=(2, 2, 2, 2))
    d = np.linalg.norm(w5["B"][-1] - w5["B"][0]) / np.linalg.norm(w5["B"][0])
    assert 1e-11 < d < 1e-8                                        # near dependence at the 1e-9 level


def test_shifts_and_seeds():
    s = synth.log_shifts(1e-4, 10.0, 12)
    assert s[0] == 1e-4 and abs(s[-1] - 10.0) < 1e-12 and np.all(np.diff(np.log(s)) > 0)
    a = synth.make_workload("w1_4x4x4x4")
    b = synth.make_workload("w1_4x4x4x4")
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["B"], b["B"])   # seeded, reproducible
