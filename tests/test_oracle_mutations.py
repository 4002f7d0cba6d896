"""Plant plausible mistakes in a copy of the oracle source (on the CPU) and check
that the pins of test_oracle_pins catch every one of them.

Each mutation is a textual edit of lbm_oracle.c compiled into a temporary
library; the oracle module is pointed at it for the duration of one check.
"""
import os
import subprocess

import pytest

import oracle as O
from oracle import build as OB
from tests import test_oracle_pins as T


def _relaxation_identity():
    T.test_cascaded_post_collision_central_moments_hit_relaxation_targets(T.OMEGA_SETS[1], True)


def _source_moments():
    T.test_source_central_moments_match_eq11()


def _streaming():
    for edges in T.EDGE_CASES:
        T.test_streaming_with_walls_brute_force(edges, (5, 3))


def _couette():
    T.test_couette_moving_wall(O.CASCADED, "north")


def _couette_east():
    T.test_couette_moving_wall(O.CASCADED, "east")


def _init():
    T.test_init_is_the_transformed_equilibrium(O.CASCADED)


def _bgk_strain():
    T.test_couette_moving_wall(O.BGK, "north")


def _conservation():
    for m in (O.CASCADED, O.BGK, O.RAWMRT):
        T.test_collision_conserves_mass_and_adds_force(m)


def _corner_symmetry():
    T.test_cavity_is_equivariant_under_a_quarter_turn(O.CASCADED)


def _strain_divergence():
    for om in ((1.3, 1.6, 1.6, 1.0, 1.0, 1.0), (1.6, 1.3, 1.3, 1.0, 1.0, 1.0)):
        T.test_strain_divergence_satisfies_continuity(O.CASCADED, om)


def _force_field():
    for m in (O.CASCADED, O.BGK, O.RAWMRT):
        T.test_force_field_adds_to_the_uniform_force(m)


def _sound_wave():
    T.test_standing_sound_wave_speed_and_damping(O.CASCADED, T.SOUND_RATES[0])


def _unit_rates():
    T.test_unit_rates_give_the_cascaded_equilibrium()


def _mrt():
    T.test_raw_mrt_relaxes_orthogonal_moments()


MUTATIONS = [
    # (name, original text, planted text, pin expected to fail)
    ("sigma_xxy central reading (dropped source term in g6)",
     "uy * kxx - 0.5 * sxxy)", "uy * kxx)", _relaxation_identity),
    ("wrong sign of g5 in f~5", "(2.0 * g3 + g5 - g6 - g7 + g8)", "(2.0 * g3 - g5 - g6 - g7 + g8)",
     _relaxation_identity),
    ("kxyy in place of kxxy in g6", "+ kxxy - 2.0 * ux * kxy", "+ kxyy - 2.0 * ux * kxy",
     _relaxation_identity),
    ("dropped F/2 in the velocity", "*ux = (jx + 0.5 * F[0]) / r;", "*ux = jx / r;", _relaxation_identity),
    ("wrong sign of m4 in S4", "(-6.0 * m2 - m3 - 9.0 * m4", "(-6.0 * m2 - m3 + 9.0 * m4", _source_moments),
    ("wrong rest target of xxyy", "(1.0 / 9.0) * rho + 3.0", "(1.0 / 3.0) * rho + 3.0", _unit_rates),
    ("lid correction with the wrong sign", "corr = 6.0 * W[b]", "corr = -6.0 * W[b]", _couette),
    ("west and east wall speeds taken along x",
     "(wall >= 2) ? L->wall_u[wall] : 0.0;\n                        const real Uy = (wall >= 2) ? 0.0 : L->wall_u[wall];",
     "L->wall_u[wall];\n                        const real Uy = 0.0;", _couette_east),
    ("start state shifted by +S/2", "f[a * plane + n] = feq[a] - 0.5 * S[a];",
     "f[a * plane + n] = feq[a] + 0.5 * S[a];", _init),
    ("BGK strain inverted with the cascaded rates", "if (L->model == ORACLE_BGK) om[0] = om[2] = om[1];",
     "", _bgk_strain),
    ("bounce-back into the same direction", "const int b = OPP[a];", "const int b = a;", _streaming),
    ("lid term on the links through a corner", "if (!corner && L->edge[wall] == ORACLE_MOVING_WALL)",
     "if (L->edge[wall] == ORACLE_MOVING_WALL)", _corner_symmetry),
    ("omega_4 in place of omega_3 in the strain divergence (Eq. 28)", "const real div = -1.5 * om[0] * n3;",
     "const real div = -1.5 * om[1] * n3;", _strain_divergence),
    ("force field replaces the uniform force", "F[0] += L->force_field[node];", "F[0] = L->force_field[node];",
     _force_field),
    ("transposed K in the raw-MRT projection", "m += KMAT[a][b] * fb[a];", "m += KMAT[b][a] * fb[a];",
     _mrt),
    ("omega_4 used for the bulk kernel", "const real g3 = (w3 / 12.0)", "const real g3 = (w4 / 12.0)",
     _sound_wave),
    ("omega_3 used for the deviatoric kernel", "(w4 / 4.0) * (rho * (ux * ux - uy * uy)",
     "(w3 / 4.0) * (rho * (ux * ux - uy * uy)", _relaxation_identity),
]


@pytest.mark.parametrize("name,orig,planted,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, planted, pin):
    src = open(OB.SRC).read()
    assert src.count(orig) == 1, f"mutation anchor not unique for {name}"
    mutant_c = tmp_path / "lbm_oracle.c"
    mutant_c.write_text(src.replace(orig, planted))
    lib = str(tmp_path / f"liblbm_oracle_mut{os.getpid()}.so")
    subprocess.run(["gcc", *OB.CFLAGS, "-I", OB.HERE, str(mutant_c), "-o", lib, "-lm"], check=True)
    pin()  # the unmutated oracle passes the pin
    with O.substituted_library(lib):
        with pytest.raises(AssertionError):
            pin()
