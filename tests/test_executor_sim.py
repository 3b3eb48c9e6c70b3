"""The executor's immediate schedule against a simulated copy engine on the
CPU (tests/executor_sim.cc): random copy and kernel durations on three
in-order streams, a copy that fails to issue, a kernel that never completes
(the wait limit must end the call with VX_E_TIMEOUT), and chunks whose every
wait stays under the limit while the whole run takes ten times longer (no
timeout).  The simulation checks every scheduling rule on every decision."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sim(tmp_path_factory):
    exe = tmp_path_factory.mktemp("sim") / "executor_sim"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-Wall", "-Werror",
                           "-I", os.path.join(ROOT, "paper_2502_09541_gb300", "csrc"),
                           "-o", str(exe), os.path.join(ROOT, "tests", "executor_sim.cc")])
    return str(exe)


@pytest.mark.parametrize("scenario", ["random", "random_deep", "copy_fails", "stuck_kernel", "slow_progress"])
@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_schedule_rules_and_failures(sim, scenario, seed):
    r = subprocess.run([sim, scenario, str(seed)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
