"""Plant plausible mistakes in a copy of the D3Q27 oracle source (on the CPU)
and check that a pin of test_oracle3d_pins catches each of them."""
import os
import subprocess

import pytest

from oracle import build as OB
from oracle import d3q27 as D
from tests import test_oracle3d_pins as T


def _relaxation():
    T.test_post_collision_central_moments_relax_to_their_targets()


def _conservation():
    T.test_collision_conserves_mass_and_gains_momentum_F()


def _symmetry():
    T.test_cubic_symmetry_of_whole_runs()


def _streaming():
    T.test_streaming_is_a_periodic_shift_of_each_population()


def _start():
    T.test_start_state_returns_the_requested_fields()


def _equilibrium():
    T.test_equilibrium_is_the_product_maxwellian()


MUTATIONS = [
    # (name, original text, planted text, pin expected to fail)
    ("trace relaxed at the shear rate", "const double Tp = T + ob * (rho - T)", "const double Tp = T + os * (rho - T)",
     _relaxation),
    ("dropped F/2 in the velocity", "u[d] = (j[d] + 0.5 * F[d]) / r;", "u[d] = j[d] / r;", _relaxation),
    ("source adds F/2", "cp[1] += F[0];", "cp[1] += 0.5 * F[0];", _conservation),
    ("order-n moments at the rate of order n - 1", "cp[m] = c[m] + om[n - 1] * (eq - c[m]);",
     "cp[m] = c[m] + om[n - 2] * (eq - c[m]);", _relaxation),
    ("xz off-diagonal moment at the bulk rate", "cp[xz] = (1.0 - os) * c[xz];", "cp[xz] = (1.0 - ob) * c[xz];",
     _symmetry),
    ("yy and zz swapped in the deviator recombination", "cp[yy] = (Tp - 2.0 * D1p + D2p) / 3.0;",
     "cp[yy] = (Tp + D1p - 2.0 * D2p) / 3.0;", _symmetry),
    ("streaming against the velocity", "const int xt = (x + e[a][0] + L->nx) % L->nx;",
     "const int xt = (x - e[a][0] + L->nx) % L->nx;", _streaming),
    ("start state shifted by +S/2", "f[idx(L, a, x, y, z)] = feq[a] - 0.5 * S[a];",
     "f[idx(L, a, x, y, z)] = feq[a] + 0.5 * S[a];", _start),
    ("second-order equilibrium moment 1/2 instead of 1/3", "static const double MEQ[3] = {1.0, 0.0, 1.0 / 3.0};",
     "static const double MEQ[3] = {1.0, 0.0, 1.0 / 2.0};", _equilibrium),
]


@pytest.mark.parametrize("name,orig,planted,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, planted, pin):
    src = open(OB.SRC3).read()
    assert src.count(orig) == 1, f"mutation anchor not unique for {name}"
    mutant_c = tmp_path / "lbm3d_oracle.c"
    mutant_c.write_text(src.replace(orig, planted))
    lib = str(tmp_path / f"liblbm3d_oracle_mut{os.getpid()}.so")
    subprocess.run(["gcc", *OB.CFLAGS, "-I", OB.HERE, str(mutant_c), "-o", lib, "-lm"], check=True)
    pin()  # the unmutated oracle passes the pin
    with D.substituted_library(lib):
        with pytest.raises(AssertionError):
            pin()
