"""The benchmark's parameter table (bench.PARAMS, plain numbers the oracle's reference arm
uses without loading the library) agrees with the library's tuner (ewald_tune at the
workload's tuning tolerance, bench.TUNE_TOL, else 1e-6; r_c fixed where bench.WORKLOADS fixes
it), so that both arms of the
benchmark evaluate the same (beta, r_c, k_max).  Host-only: the tuner launches nothing."""
import math

import pytest

import bench


def test_parameter_table_matches_the_tuner():
    from paper_1708_01135_gb300 import ewald as E
    try:
        E.lib()
    except RuntimeError as e:     # not built in this checkout
        pytest.skip(str(e))
    sizes = {"random_32768": (32768, 32.0), "rocksalt_262144": (262144, 64.0),
             "random_2097152": (2097152, 128.0)}
    for name, (n, L) in sizes.items():
        rc_fixed = bench.WORKLOADS[name][1]
        rc, beta, km = E.tune(n, L, bench.TUNE_TOL.get(name, bench.TOL), r_c=rc_fixed)
        prc, pbeta, pkm = bench.PARAMS[name]
        assert rc == prc and km == pkm and math.isclose(beta, pbeta, rel_tol=1e-14), name


def test_converged_reference_parameters():
    # both truncation errors ~exp(-p^2) at p = 4.3 (~1e-8), r_c at the minimum-image limit
    rc, beta, km = bench.converged_params(128.0)
    assert rc == 64.0 and math.isclose(beta * rc, 4.3)
    assert km == math.ceil(4.3 * beta * 128.0 / math.pi)
    assert math.exp(-(math.pi * km / (beta * 128.0)) ** 2) < 1e-8
