"""The hand-run checking scripts still run (CPU): one planted slip per target
of tests/plant_slips.py, and tests/proposal_ceiling.py on one image."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plant_slips_runs_one_slip_per_target():
    r = subprocess.run([sys.executable, "tests/plant_slips.py", "c", "proposal", "scfv", "resize", "parity",
                        "--only", "lap_sign", "input_shift_127", "pca_plus_mean", "round_floor", "dup_record_margin"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("CAUGHT") == 5, r.stdout


def test_proposal_ceiling_runs():
    r = subprocess.run([sys.executable, "tests/proposal_ceiling.py", "1", "1"], cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "out of detection" in r.stdout
