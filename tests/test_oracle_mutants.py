"""Mutation check of the oracle's pins.

Each mutant build of oracle.c plants one plausible mistake (ORACLE_MUTANT = n):
  1 dimer propensity without the 1/2          2 second reactant index replaced by the first
  3 waiting time without the internal time     4 first channel that can fire wins (no minimum)
  5 internal times advanced with post-event a  6 internal times advanced by a * t, not a * dt
  7 consumption applied with the wrong sign    8 refresh replaces P instead of adding to it
  9 refresh reuses the first draw of a channel 10 grid sampled after instead of before events
 11 likelihood with the integral's sign flipped 12 logarithm series truncated after two terms
 13 uniform mapping that can produce u = 0      14 Philox round mixing the wrong word
In the absolute-time form (mode 1):
 15 touched channels' internal times not brought up to the event (other than the fired one)
 16 dependency test reads only a reaction's first reactant species
 17 absolute firing time computed without the update time (a relative waiting time)
 18 internal times not brought up to the end of the run
In Table 3's rescaled form (mode 2):
 19 waiting times shifted by dt but not rescaled by p_k / a_k
 20 the fired channel's new waiting time reuses its previous draw
 21 a frozen channel's remaining internal time lost when it resumes
With time-dependent rates c_k (1 + beta_k t):
 22 the internal-time integral without its beta dt^2 / 2 term
 23 waiting times solved with the rate at time 0 instead of at the current time
 24 ln a_mu taken at the previous event's time
The pin suite (tests/test_oracle_pins.py) must fail on every one of them.
"""
import concurrent.futures
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
MUTANTS = list(range(1, 25))


def _run_pins(n, tmpdir):
    lib = os.path.join(tmpdir, "liboracle_mut%d.so" % n)
    oracle.build(force=True, out=lib, extra_flags=["-DORACLE_MUTANT=%d" % n])
    env = dict(os.environ, ORACLE_LIB=lib, ORACLE_THREADS="2")
    # a mutant may also make a pin's simulation run away: the per-test timeout counts as a failure
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"), "-x", "-q",
                        "-p", "no:cacheprovider", "--timeout=20", "--timeout-method=thread"], env=env,
                       capture_output=True, text=True, timeout=300)
    return n, r.returncode, r.stdout[-400:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    pytest.importorskip("pytest_timeout")
    # control: the unmodified oracle built the same way passes the same harness
    n, rc, out = _run_pins(0, str(tmp_path))
    assert rc == 0, out
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, (os.cpu_count() or 2) // 2)) as ex:
        results = list(ex.map(lambda n: _run_pins(n, str(tmp_path)), MUTANTS))
    survivors = [(n, out) for n, rc, out in results if rc == 0]
    assert not survivors, survivors
