"""The oracle's pins catch plausible mistakes: each test plants one mistake in
the oracle (monkeypatched, on the CPU) and checks that a pin of
test_oracle_collision / test_oracle_physics / test_oracle_nested now fails."""
import math

import pytest
import torch

import oracle.collision as C
import oracle.lattice as Lat
import oracle.solver as S
from tests import test_oracle_collision as TC
from tests import test_oracle_lattice as TL
from tests import test_oracle_nested as TN
from tests import test_oracle_physics as TP


def plant(monkeypatch, module, name, new):
    """Replace an oracle function, also where a test module imported it by name."""
    old = getattr(module, name)
    monkeypatch.setattr(module, name, new)
    for m in (TC, TL, TN, TP):
        if getattr(m, name, None) is old:
            monkeypatch.setattr(m, name, new)


def fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def test_wrong_sign_in_a_velocity_is_caught(monkeypatch):
    bad = list(Lat._D3Q19[1])
    bad[9] = -bad[9]                      # e_9 = (1, -1, 0) -> (1, 1, 0)
    monkeypatch.setattr(Lat, "_D3Q19", (Lat._D3Q19[0], tuple(bad), Lat._D3Q19[2]))
    assert fails(TL.test_velocity_set_shape, 19)


def test_wrong_weight_is_caught(monkeypatch):
    monkeypatch.setattr(Lat, "_W27", {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 108})
    assert fails(TL.test_weights_float_match_exact, 27)


def test_dropped_quadratic_term_in_equilibrium_is_caught(monkeypatch):
    orig = C.feq_incompressible

    def feq(drho, u, Q=19):
        e = Lat.velocities(Q).to(C.DTYPE)
        w = Lat.weights(Q)
        eu = e @ u
        return w[:, None] * (drho[None] + 3.0 * eu - 1.5 * (u * u).sum(0)[None])
    plant(monkeypatch, C, "feq_incompressible", feq)
    assert fails(TP.test_shear_wave_viscosity, "d3q19", 1.2) or fails(TC.test_mrt_shear_projection_closed_form)


def test_transposed_mrt_row_is_caught(monkeypatch):
    orig = C.mrt_matrix

    def M():
        m = orig().clone()
        m[[4, 9]] = m[[9, 4]]             # shear row mu12 swapped with the trace row
        return m
    plant(monkeypatch, C, "mrt_matrix", M)
    assert fails(TC.test_mrt_shear_projection_closed_form)


def test_wrong_smagorinsky_factor_is_caught(monkeypatch):
    plant(monkeypatch, C, "tau_total",
          lambda tau0, cs, Qn: tau0 + (torch.sqrt(tau0 * tau0 + 9.0 * cs * cs * Qn) - tau0) / 2.0)
    assert fails(TC.test_smagorinsky_tau_solves_quadratic)


def test_pre_collision_moments_in_cascade_are_caught(monkeypatch):
    orig = C.fclb_relax

    def relax(kappa, omega, rho, force=None):
        out = orig(kappa, omega, rho, force)
        k = kappa
        out[:, C.IDX[(2, 2, 0)]] = k[:, C.IDX[(2, 0, 0)]] * k[:, C.IDX[(0, 2, 0)]]   # pre instead of post
        return out
    plant(monkeypatch, C, "fclb_relax", relax)
    assert fails(TC.test_fclb_conserves_and_fixed_point) or fails(TP.test_shear_wave_viscosity, "d3q27", 1.8) \
        or fails(TC.test_fclb_second_order_relaxation) or fails(TC.test_fclb_omega_one_gives_product_equilibrium)


def test_transposed_central_moment_matrix_is_caught(monkeypatch):
    orig = C.central_moment_matrix
    plant(monkeypatch, C, "central_moment_matrix", lambda u: orig(u).transpose(1, 2).contiguous())
    assert fails(TC.test_central_moments_match_table2_polynomials)


def test_missing_interface_rescaling_is_caught(monkeypatch):
    monkeypatch.setattr(S.NestedSolver, "_taus_cf", lambda self, l, S_c: (S_c * 0 + 2.0, S_c * 0 + 3.0))
    assert fails(TN.test_shear_wave_stress_crosses_interfaces, "d3q19")


def _weighted_c2f(monkeypatch, w):
    """Plant F_1 = (1 - w) f~(t) + w f~(t+1) for the second fine substep."""
    orig = S.NestedSolver._c2f

    def c2f(self, l, s, old, new, oldS, newS):
        if s == 0:
            return orig(self, l, 0, old, new, oldS, newS)
        mix, mixS = (1 - w) * old + w * new, (1 - w) * oldS + w * newS
        return orig(self, l, 0, mix, mix, mixS, mixS)
    monkeypatch.setattr(S.NestedSolver, "_c2f", c2f)


@pytest.mark.parametrize("w", [0.0, 0.4, 0.6, 1.0])
def test_wrong_temporal_weight_is_caught(monkeypatch, w):
    """Old-only (0), new-only (1) and a slightly wrong weight (0.4, 0.6)
    each break the closed-form phase speed of the drifting wave."""
    _weighted_c2f(monkeypatch, w)
    assert fails(TN.test_drifting_wave_crosses_interfaces_at_the_exact_phase_speed, 0.05)


def test_new_only_temporal_interpolation_on_both_substeps_is_caught(monkeypatch):
    orig = S.NestedSolver._c2f

    def c2f(self, l, s, old, new, oldS, newS):
        return orig(self, l, 0, new, new, newS, newS)   # always the new coarse values
    monkeypatch.setattr(S.NestedSolver, "_c2f", c2f)
    assert fails(TN.test_drifting_wave_crosses_interfaces_at_the_exact_phase_speed, 0.05)


def test_wrong_inflow_velocity_is_caught(monkeypatch):
    orig = S.NestedSolver._apply_bc

    def bc(self, l, sub):
        self.inflow = dict(self.inflow, perturb=0.02)
        return orig(self, l, sub)
    monkeypatch.setattr(S.NestedSolver, "_apply_bc", bc)
    assert fails(TN.test_inflow_ghosts_carry_disc_velocity, "d3q19")


def test_bounce_back_without_reversal_is_caught(monkeypatch):
    """A no-slip wall that returns the incoming population itself instead of
    its opposite (no momentum reversal)."""
    from tests import test_oracle_walls as TW
    orig = S.NestedSolver._vel_index

    def idx(self, ex, ey, ez):
        return orig(self, -ex, -ey, -ez) if (ex, ey, ez) != (0, 0, 0) else orig(self, 0, 0, 0)

    def wall_pulls(self, f, pre):
        # bounce-back reads f_i instead of f_opp(i): flip the lookup only there
        monkeypatch.setattr(S.NestedSolver, "_vel_index", idx)
        try:
            S_orig_wall(self, f, pre)
        finally:
            monkeypatch.setattr(S.NestedSolver, "_vel_index", orig)
    S_orig_wall = S.NestedSolver._wall_pulls
    monkeypatch.setattr(S.NestedSolver, "_wall_pulls", wall_pulls)
    assert fails(TW.test_no_slip_poiseuille_profile)
    assert fails(TW.test_x_walls_hold_poiseuille_profile)
    assert fails(TW.test_shear_mode_between_no_slip_walls_decays_at_the_channel_rate, "d3q19", 3, 0)


def test_free_slip_flipping_the_tangential_component_is_caught(monkeypatch):
    """A free-slip wall that mirrors the wrong velocity component."""
    from tests import test_oracle_walls as TW
    orig = S.NestedSolver._vel_index

    def wall_pulls(self, f, pre):
        def idx(s, ex, ey, ez):
            return orig(s, -ex, ey, ez) if ex != 0 else orig(s, ex, ey, ez)
        monkeypatch.setattr(S.NestedSolver, "_vel_index", idx)
        try:
            orig_wall(self, f, pre)
        finally:
            monkeypatch.setattr(S.NestedSolver, "_vel_index", orig)
    orig_wall = S.NestedSolver._wall_pulls
    monkeypatch.setattr(S.NestedSolver, "_wall_pulls", wall_pulls)
    assert fails(TW.test_free_slip_keeps_tangential_uniform_flow, "d3q27")


def _plant_outlet(monkeypatch, ghost):
    monkeypatch.setattr(S.NestedSolver, "_outlet_ghost", ghost)


def test_outlet_without_non_equilibrium_part_is_caught(monkeypatch):
    """A pressure outlet that keeps only the equilibrium at rho_out."""
    from tests import test_oracle_outlet as TO

    def ghost(self, src):
        rl = torch.full_like(src[0], self.rho_out - 1.0 if self.m.name == "d3q19" else self.rho_out)
        return self.m.feq(rl, self.m.velocity(src))
    _plant_outlet(monkeypatch, ghost)
    assert fails(TO.test_outlet_cell_of_x_invariant_state_evolves_as_periodic, "d3q27")
    assert fails(TO.test_outlet_ghost_has_outlet_density_and_cell_velocity, "d3q19")


def test_outlet_that_copies_the_cell_is_caught(monkeypatch):
    """A 'pressure' outlet that is the zero-gradient copy (rho_out unused)."""
    from tests import test_oracle_outlet as TO
    _plant_outlet(monkeypatch, lambda self, src: src.clone())
    assert fails(TO.test_outlet_drains_overpressure_to_rho_out, "d3q27")
    assert fails(TO.test_outlet_ghost_has_outlet_density_and_cell_velocity, "d3q27")


def test_outlet_with_the_density_correction_reversed_is_caught(monkeypatch):
    from tests import test_oracle_outlet as TO

    def ghost(self, src):
        u = self.m.velocity(src)
        rl_n = self.m.density_like(src)
        rl = torch.full_like(rl_n, self.rho_out - 1.0 if self.m.name == "d3q19" else self.rho_out)
        return src - (self.m.feq(rl, u) - self.m.feq(rl_n, u))
    _plant_outlet(monkeypatch, ghost)
    assert fails(TO.test_outlet_ghost_has_outlet_density_and_cell_velocity, "d3q19")
    assert fails(TO.test_outlet_drains_overpressure_to_rho_out, "d3q27")


def test_bouzidi_with_q_fixed_at_one_half_is_caught(monkeypatch):
    """Interpolated walls treated as half-way bounce-back (q ignored)."""
    from oracle import nozzle as N
    from tests import test_oracle_nozzle as TZ
    orig = N.Body.wall_values

    def wall_values(self, f):
        q = self.q
        self.q = torch.full_like(q, 0.5)
        try:
            return orig(self, f)
        finally:
            self.q = q
    monkeypatch.setattr(N.Body, "wall_values", wall_values)
    assert fails(TZ.test_plane_walls_at_any_position_hold_poiseuille, 2.3, 5.2)
    assert fails(TZ.test_shear_wave_between_interpolated_walls_decays_at_the_true_width, "d3q19", 2.3, 5.2)


def test_bouzidi_with_one_branch_for_all_q_is_caught(monkeypatch):
    """The q < 1/2 interpolation used for every link (an extrapolation for
    q > 1/2)."""
    from oracle import nozzle as N
    from tests import test_oracle_nozzle as TZ

    def wall_values(self, f):
        a = f[self.i, self.f_idx[0], self.f_idx[1], self.f_idx[2]]
        b = f[self.i, self.s_idx[0], self.s_idx[1], self.s_idx[2]]
        return torch.where(self.has2, 2.0 * self.q * a + (1.0 - 2.0 * self.q) * b, a)
    monkeypatch.setattr(N.Body, "wall_values", wall_values)
    assert fails(TZ.test_plane_walls_at_any_position_hold_poiseuille, 2.3, 5.2)


def test_cap_inflow_with_the_wrong_density_cell_is_caught(monkeypatch):
    """The cap's inflow equilibrium taking the density of the solid cell
    instead of the fluid cell downstream."""
    from tests import test_oracle_nozzle as TZ
    orig = S.NestedSolver._body_links

    def links(self, l, sub):
        b = self.body
        if b is None:
            return orig(self, l, sub)
        keep = b.b_idx
        f = self.f[l]
        # shift the index the cap rule adds one to: reads x_b itself
        b.b_idx = (keep[0], keep[1], keep[2] - b.inflow.long())
        try:
            orig(self, l, sub)
        finally:
            b.b_idx = keep
    monkeypatch.setattr(S.NestedSolver, "_body_links", links)
    assert fails(TZ.test_cap_inflow_equals_face_inflow, "d3q27")


def test_half_width_at_half_maximum_is_caught(monkeypatch):
    """A spreading width taken where u falls to u_m / 2 instead of u_m / e."""
    import types
    import oracle.jetstats as J
    from tests import test_oracle_jetstats as TJ
    fake = types.SimpleNamespace(**{k: getattr(math, k) for k in dir(math) if not k.startswith("_")})
    fake.e = 2.0
    monkeypatch.setattr(J, "math", fake)
    assert fails(TJ.test_gaussian_profile_gives_its_width_and_unit_fit)
    assert fails(TJ.test_parabolic_profile_half_width_closed_form)


def test_bouzidi_fraction_from_the_solid_side_is_caught(monkeypatch):
    """The wall fraction measured from the solid cell (1 - q instead of q)."""
    from oracle import nozzle as N
    from tests import test_oracle_nozzle as TZ
    orig = N.Body.wall_values

    def wall_values(self, f):
        q = self.q
        self.q = 1.0 - q
        try:
            return orig(self, f)
        finally:
            self.q = q
    monkeypatch.setattr(N.Body, "wall_values", wall_values)
    assert fails(TZ.test_plane_walls_at_any_position_hold_poiseuille, 2.3, 5.2)
    assert fails(TZ.test_plane_walls_at_any_position_hold_poiseuille, 1.6, 4.45)
