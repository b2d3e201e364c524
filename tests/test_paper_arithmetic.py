"""The paper's printed figures and the arithmetic that defines the reported metrics.

The real-time factor (Table 'Performance statistics' caption) is the substep length over
the frame time, scaled by the number of parallel environments.  bench.py reports it with
this definition; the rows below pin the definition to the paper's own numbers."""
import json
import os

import pytest

with open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")) as f:
    PAPER = json.load(f)


def real_time_factor(envs, substeps, frame_ms, dt=1.0 / 60.0):
    """(dt / substeps) / frame time x envs -- as the paper's table caption defines it."""
    return (dt / substeps) / (frame_ms * 1e-3) * envs


@pytest.mark.parametrize("scene", list(k for k in PAPER["performance"] if not k.startswith("_")))
def test_real_time_factor_reproduces_table(scene):
    r = PAPER["performance"][scene]
    assert real_time_factor(r["envs"], r["substeps"], r["time_ms"]) == pytest.approx(r["real_time"], rel=0.02)


def test_frame_time_is_handling_plus_solution():
    for k in ("peg_in_hole", "nut_and_bolt", "dsub_connector", "gear_assembly"):
        c, p = PAPER["contact_statistics"][k], PAPER["performance"][k]
        assert c["handling_ms"] + c["solution_ms"] == pytest.approx(p["time_ms"])


def test_bandwidth_model_arithmetic():
    b = PAPER["bandwidth_model"]
    per_step = b["m4_contacts_before"] * b["bytes_contact_constraints"]          # 2.56 MB
    per_frame = per_step * b["jacobi_substeps"] * b["jacobi_iters"]
    assert per_frame / 1e9 == pytest.approx(b["jacobi_before_gb_per_frame"], rel=0.03)
    after = b["m4_contacts_after"] * b["bytes_contact_constraints"] * b["jacobi_substeps"] * b["jacobi_iters"]
    assert after / 1e6 == pytest.approx(b["jacobi_after_mb_per_frame"], rel=0.03)
