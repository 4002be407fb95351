"""The oracle's pins against planted mistakes (CPU).

A pin is only worth something if a plausible mistake in the function it
checks makes it fail.  Each case below copies the oracle into a scratch
directory, plants one mistake in the copy (a textual edit of one line: a
sign, a factor, an index, a direction, a dropped term), and runs the pin
files that cover that function against the copy in a separate interpreter.
The case passes when that run ends with failing tests (pytest exit code 1);
an unmodified copy must pass the same files (exit code 0), which shows that
the harness itself does not cause the failures.  Edits that cannot change
any result are not listed: for instance, dropping the second hop of the
coalescence trace in `layout.multires_interface` leaves the classification
as it is, since that hop always lands in the coarse voxel G - c_i, which the
first hop of another subcell of G reaches as well, and levels own whole
coarse voxels.

The product is not involved: only `oracle/`, the input generators of
`paper_2503_07898_gb300/workloads.py` and the `-m "not gpu"` pin files are
copied.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PINS = "test_oracle_pins.py"
Q27 = "test_oracle_d3q27.py"
MR = "test_oracle_multires.py"
CL = "test_oracle_closure.py"

# (name, oracle file, original text, planted text, pin files run)
MUTATIONS = [
    # lattice: weights, equilibrium, regularized projection, velocity order
    ("weights_axis_edge_swapped", "lattice.py",
     "_W19 = [Fraction(1, 3)] + [Fraction(1, 18)] * 6 + [Fraction(1, 36)] * 12",
     "_W19 = [Fraction(1, 3)] + [Fraction(1, 36)] * 6 + [Fraction(1, 18)] * 12", [PINS]),
    ("equilibrium_quadratic_factor", "lattice.py",
     "1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq", "1.0 + 3.0 * cu + 4.0 * cu * cu - 1.5 * usq",
     [PINS]),
    ("equilibrium_usq_sign", "lattice.py",
     "1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq", "1.0 + 3.0 * cu + 4.5 * cu * cu + 1.5 * usq",
     [PINS]),
    ("regularized_projection_factor", "lattice.py",
     "out[i] = 4.5 * self.W[i] * acc", "out[i] = 3.0 * self.W[i] * acc", [PINS]),
    ("regularized_projection_trace_dropped", "lattice.py",
     "(1.0 / 3.0 if a == b else 0.0)", "(0.0 if a == b else 0.0)", [PINS]),
    ("velocity_order_not_paired", "lattice.py",
     "(1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),",
     "(1, 1, 0), (1, -1, 0), (-1, -1, 0), (-1, 1, 0),", [PINS]),
    # single-resolution step: streaming, walls, collision, regularized nodes
    ("stream_direction_reversed", "lbm.py",
     "src_val = _shift(f[i], cz, cy, cx)", "src_val = _shift(f[i], -cz, -cy, -cx)", [PINS]),
    ("bounce_back_not_opposite", "lbm.py",
     "g[i] = np.where(wall, f[lat.OPP[i]], src_val)", "g[i] = np.where(wall, f[i], src_val)",
     [PINS]),
    ("outside_voxels_not_walls", "lbm.py",
     "wall = (src_type == SOLID) | (src_type == OUTSIDE)", "wall = (src_type == SOLID)", [PINS]),
    ("box_side_one_end_only", "lbm.py",
     "out = out | (s < 0) | (s >= n)", "out = out | (s < 0)", [PINS]),
    ("bgk_rate_inverted", "lbm.py",
     "f_star = g - (g - feq) / tau", "f_star = g - (g - feq) * tau", [PINS]),
    ("reg_collision_factor", "lbm.py",
     "f_star = feq + (1.0 - 1.0 / tau) * lat.regularized_neq(lat.second_moment(g - feq))",
     "f_star = feq + (1.0 - 0.5 / tau) * lat.regularized_neq(lat.second_moment(g - feq))", [PINS]),
    ("velocity_node_density_sign", "lbm.py",
     "rho = s / (1.0 + un)", "rho = s / (1.0 - un)", [PINS]),
    ("pressure_node_velocity_sign", "lbm.py",
     "un = s / rho - 1.0", "un = 1.0 - s / rho", [PINS]),
    ("known_sum_factor_dropped", "lbm.py",
     "s = g_node[k0].sum(axis=0) + 2.0 * g_node[kp].sum(axis=0)",
     "s = g_node[k0].sum(axis=0) + g_node[kp].sum(axis=0)", [PINS]),
    ("unknown_neq_bounce_sign", "lbm.py",
     "g[i] = feq[i] + (g[j] - feq[j])", "g[i] = feq[i] - (g[j] - feq[j])", [PINS]),
    # D3Q27 corner weights
    ("d3q27_corner_weight", "lattice.py",
     "[Fraction(1, 54)] * 12 + [Fraction(1, 216)] * 8", "[Fraction(1, 54)] * 12 + [Fraction(1, 108)] * 8",
     [Q27]),
    # multi-resolution exchange
    ("level_tau_scaling_inverted", "multires.py",
     "return 0.5 + (tau0 - 0.5) / (2 ** level)", "return 0.5 + (tau0 - 0.5) * (2 ** level)", [MR]),
    ("explosion_substeps_swapped", "multires.py",
     "                if k == 1:\n", "                if k == 2:\n", [MR]),
    ("coalescence_second_hop_dropped", "multires.py",
     "coal = subcell_mean(shift(held, c))", "coal = subcell_mean(held)", [MR]),
    ("coalescence_reads_start_state", "multires.py",
     "held = np.where(own_f == lv - 1, f1_fine[i], v1)",
     "held = np.where(own_f == lv - 1, f0_fine[i], v1)", [MR]),
    ("volume_weight_wrong", "multires.py",
     "out += (8.0 ** lv) * lbm.conservation(self.f[lv])",
     "out += (4.0 ** lv) * lbm.conservation(self.f[lv])", [MR]),
    # layout tables
    ("morton_y_bit_misplaced", "layout.py",
     "code |= ((by >> k) & 1) << (3 * k + 1)", "code |= ((by >> k) & 1) << (3 * k)", [PINS]),
    ("boundary_blocks_last", "layout.py",
     "keys = [(0 if isb else 1, morton_code(*c)) for c, isb in zip(active, boundary)]",
     "keys = [(1 if isb else 0, morton_code(*c)) for c, isb in zip(active, boundary)]", [PINS]),
    ("interface_explosion_source_reversed", "layout.py",
     "dep |= at(o, C[i], 1) == lv + 1", "dep |= at(o, C[i], -1) == lv + 1", [MR]),
    # learned closure: network, training, features, data path
    ("relu_derivative_dropped", "closure.py",
     "dz2 = dh2 * (z2 > 0)", "dz2 = dh2", [CL]),
    ("adam_bias_correction_dropped", "closure.py",
     "mhat = m / (1 - beta1 ** step)", "mhat = m", [CL]),
    ("fold_bias_sign", "closure.py",
     'p["b1"] = p["b1"] - p["W1"] @ (mu / sd)', 'p["b1"] = p["b1"] + p["W1"] @ (mu / sd)', [CL]),
    ("splitmix_final_shift", "closure.py",
     "return x ^ (x >> 31)", "return x ^ (x >> 30)", [CL]),
    ("feature_scale", "closure.py",
     "s = rho / 3.0", "s = rho / 2.0", [CL]),
    ("eddy_central_difference_reversed", "closure.py",
     "0.5 * (np.roll(ub[b], -1, axis=axis) - np.roll(ub[b], 1, axis=axis))",
     "0.5 * (np.roll(ub[b], 1, axis=axis) - np.roll(ub[b], -1, axis=axis))", [CL]),
    ("eddy_sign", "closure.py",
     "nu_t = np.where(den > 0, -num / den, 0.0)", "nu_t = np.where(den > 0, num / den, 0.0)", [CL]),
    ("eddy_factor_three_dropped", "closure.py",
     "return np.clip(3.0 * nu_t,", "return np.clip(nu_t,", [CL]),
    ("eddy_density_dropped", "closure.py",
     "den = 2.0 * rb * den", "den = 2.0 * den", [CL]),
    ("coarse_pull_shift_reversed", "closure.py",
     "out[i] = np.roll(fb[i], shift=(cz, cy, cx), axis=(0, 1, 2))",
     "out[i] = np.roll(fb[i], shift=(-cz, -cy, -cx), axis=(0, 1, 2))", [CL]),
    ("box_filter_transposed", "closure.py",
     "b = a.reshape(*lead, nz // r, r, ny // r, r, nx // r, r)",
     "b = a.reshape(*lead, r, nz // r, r, ny // r, r, nx // r)", [CL]),
    ("features_third_order_weight_sign", "closure.py",
     "w = Cf[:, a] * (Cf[:, b] ** 2 + Cf[:, c] ** 2)", "w = Cf[:, a] * (Cf[:, b] ** 2 - Cf[:, c] ** 2)",
     [CL]),
    ("features_norm_cross_factor", "closure.py",
     "pzz ** 2 + 2 * (pxy ** 2 + pxz ** 2 + pyz ** 2)", "pzz ** 2 + (pxy ** 2 + pxz ** 2 + pyz ** 2)",
     [CL]),
    ("features_trace_sign", "closure.py", "tr = pxx + pyy + pzz", "tr = pxx + pyy - pzz", [CL]),
    ("forward_bias_dropped", "closure.py",
     'z1 = X @ p["W1"].T + p["b1"]', 'z1 = X @ p["W1"].T', [CL]),
    ("gradient_w1_sign", "closure.py", 'g["W1"] = dz1.T @ X', 'g["W1"] = -dz1.T @ X', [CL]),
    ("adam_second_moment_not_squared", "closure.py",
     "v = beta2 * v + (1 - beta2) * grad * grad", "v = beta2 * v + (1 - beta2) * abs(grad)", [CL]),
    ("sgs_stress_density_dropped", "closure.py",
     "- rb * ub[a] * ub[b]", "- ub[a] * ub[b]", [CL]),
    ("strain_not_symmetrised", "closure.py",
     "S = 0.5 * (grad + grad.transpose(1, 0, *range(2, grad.ndim)))", "S = grad", [CL]),
    ("stress_deviator_dropped", "closure.py",
     "dev = tsgs[a, b] - (tr if a == b else 0.0)", "dev = tsgs[a, b]", [CL]),
    ("neighbourhood_sum_self_only", "closure.py",
     "    for dz in (-1, 0, 1):\n        for dy in (-1, 0, 1):\n            for dx in (-1, 0, 1):\n"
     "                out = out + np.roll(a",
     "    for dz in (0,):\n        for dy in (-1, 0, 1):\n            for dx in (-1, 0, 1):\n"
     "                out = out + np.roll(a", [CL]),
    ("closure_tau_not_clamped", "closure.py",
     "tau_eff[fluid] = np.maximum(tau + d_tau, TAU_MIN)", "tau_eff[fluid] = tau + d_tau", [CL]),
    ("minibatch_counter_offset", "closure.py",
     "c0 = (step - 1) * batch", "c0 = step * batch", [CL]),
    ("standardisation_constant_rule_dropped", "closure.py",
     "sd = np.where((sd > 1e-6 * np.abs(mu)) & (sd > 1e-30), sd, 1.0)",
     "sd = np.where(sd > 1e-30, sd, 1.0)", [CL]),
    ("block_activity_counts_solids", "layout.py",
     "UPDATED_TYPES = (0, 2, 3)", "UPDATED_TYPES = (0, 1, 2, 3)", [PINS]),
    ("block_neighbours_not_wrapped", "layout.py",
     "q[a] %= dims_b[a]", "q[a] = -1", [PINS]),
    ("bitmask_bit_order_reversed", "layout.py",
     "words[b // 32] |= np.uint32(1 << (b % 32))", "words[b // 32] |= np.uint32(1 << (31 - b % 32))",
     [PINS]),
    ("regularized_node_relaxation_factor", "lbm.py",
     "f_star = feq + (1.0 - 1.0 / tau) * fneq", "f_star = feq + (1.0 - 0.5 / tau) * fneq", [PINS]),
    ("taylor_green_viscosity_closed_form", "lbm.py",
     "nu = (tau - 0.5) / 3.0", "nu = (tau - 0.5) / 6.0", [PINS]),
    ("subcell_mean_pairs_wrong", "multires.py",
     "a = 0.5 * (a[..., 0::2] + a[..., 1::2])", "a = 0.5 * (a[..., 0::2] + a[..., 0::2])", [MR]),
    ("explosion_second_substep_one_hop", "multires.py",
     "ex = np.where(shift(own, c, 2) == lv, shift(f0_self[i], c, 2),",
     "ex = np.where(shift(own, c, 2) == lv, shift(f0_self[i], c, 1),", [MR]),
    ("closure_on_finest_level", "multires.py",
     "if self.theta is not None and lv > 0:", "if self.theta is not None and lv >= 0:", [MR]),
    ("explosion_opposite_population", "multires.py",
     "c_up = upsample(self.f[lv + 1][i])", "c_up = upsample(self.f[lv + 1][self.lat.OPP[i]])", [MR]),
    ("d3q27_corner_order_not_paired", "lattice.py",
     "(1, -1, 1), (-1, 1, -1), (-1, 1, 1), (1, -1, -1),",
     "(1, -1, 1), (-1, 1, 1), (-1, 1, -1), (1, -1, -1),", [Q27]),
    ("d3q27_edge_weight", "lattice.py",
     "[Fraction(2, 27)] * 6 + [Fraction(1, 54)] * 12", "[Fraction(2, 27)] * 6 + [Fraction(1, 27)] * 12",
     [Q27]),
    ("flag_normal_bits_shifted", "lbm.py",
     "return (flags >> 3) & 7", "return (flags >> 4) & 7", [PINS]),
    ("box_sides_axes_swapped", "lbm.py",
     "for coord, n, ci, per in ((x, nx, c[0], periodic[0]), (y, ny, c[1], periodic[1]),",
     "for coord, n, ci, per in ((x, nx, c[0], periodic[2]), (y, ny, c[1], periodic[1]),", [PINS]),
    ("moments_velocity_not_divided", "lattice.py", "return rho, j / rho", "return rho, j", [PINS]),
    ("second_moment_index", "lattice.py",
     "out[a, b] = np.tensordot(Cf[:, a] * Cf[:, b], f, axes=(0, 0))",
     "out[a, b] = np.tensordot(Cf[:, a] * Cf[:, a], f, axes=(0, 0))", [PINS]),
    ("known_set_reversed", "lbm.py",
     "kp = np.flatnonzero(cn > 0)", "kp = np.flatnonzero(cn < 0)", [PINS]),
    ("boundary_stress_not_neq", "lbm.py",
     "pi_neq = lat.second_moment(g - feq)", "pi_neq = lat.second_moment(g)", [PINS]),
    ("regularized_voxels_not_stored", "lbm.py",
     "updated = (types == FLUID) | reg", "updated = (types == FLUID)", [PINS]),
    ("guo_half_force_shift", "lbm.py",
     "j = j + 0.5 * np.asarray(force", "j = j + 1.0 * np.asarray(force", [PINS]),
    ("guo_source_prefactor", "lbm.py",
     "f_star[i] = f_star[i] + (1.0 - 0.5 / tau) * lat.W[i] * src",
     "f_star[i] = f_star[i] + (1.0 - 1.0 / tau) * lat.W[i] * src", [PINS]),
    ("init_skips_velocity_nodes", "lbm.py",
     "f = L.equilibrium(rho, u, q)\n    if flags is not None:\n        t = flag_type(flags)\n"
     "        upd = (t == FLUID) | (t == VELOCITY) | (t == PRESSURE)",
     "f = L.equilibrium(rho, u, q)\n    if flags is not None:\n        t = flag_type(flags)\n"
     "        upd = (t == FLUID) | (t == PRESSURE)", [PINS]),
    ("finer_neighbour_level", "multires.py",
     "finer |= nb == lv - 1", "finer |= nb == lv + 1", [MR]),
    ("level_tau_off_by_one", "multires.py",
     "tau = tau_of_level(self.tau0, lv)", "tau = tau_of_level(self.tau0, lv + 1)", [MR]),
    ("finest_solids_updated", "multires.py",
     "            mine = mine & self.updated0\n        self.f[lv] = np.where",
     "            mine = mine\n        self.f[lv] = np.where", [MR]),
    ("coalescence_first_hop_state", "multires.py",
     "v1 = np.where(shift(own_f, c) == lv - 1, shift(f0_fine[i], c), shift(s_up, c))",
     "v1 = np.where(shift(own_f, c) == lv - 1, shift(f1_fine[i], c), shift(s_up, c))", [MR]),
    ("loss_gradient_factor", "closure.py", "dy = 2.0 * r / n", "dy = r / n", [CL]),
    ("bias_gradient_mean", "closure.py",
     'g["b2"] = dz2.sum(axis=0)', 'g["b2"] = dz2.mean(axis=0)', [CL]),
    ("relu_as_abs", "closure.py", "h2 = np.maximum(z2, 0.0)", "h2 = np.abs(z2)", [CL]),
    ("fold_output_scale", "closure.py",
     'p["W3"] = p["W3"] * y_sd', 'p["W3"] = p["W3"] / y_sd', [CL]),
    ("standardisation_sample_deviation", "closure.py",
     "mu, sd = X.mean(axis=0), X.std(axis=0)", "mu, sd = X.mean(axis=0), X.std(axis=0, ddof=1)", [CL]),
    ("filtered_velocity_undivided", "closure.py", "ub = jb / rb", "ub = jb", [CL]),
    ("gradient_axis_mapping", "closure.py", "axis = 2 - a ", "axis = a ", [CL]),
    ("target_upper_clamp", "closure.py",
     "np.clip(3.0 * nu_t, -(tau_coarse - 0.5) + 1e-3, 0.5)",
     "np.clip(3.0 * nu_t, -(tau_coarse - 0.5) + 1e-3, 0.25)", [CL]),
    ("tau_feature_shifted", "closure.py",
     "tau_f = np.full(rho.shape, float(tau))", "tau_f = np.full(rho.shape, float(tau) - 0.5)", [CL]),
    ("pressure_blocks_not_boundary", "layout.py",
     "REGULARIZED_TYPES = (2, 3)", "REGULARIZED_TYPES = (2,)", [PINS]),
    ("coarse_neighbour_axes_swapped", "layout.py",
     "xc[b, k] = bmaps[lv + 1][(q[0] // 2, q[1] // 2, q[2] // 2)]",
     "xc[b, k] = bmaps[lv + 1].get((q[1] // 2, q[0] // 2, q[2] // 2), -2)", [PINS]),
    ("features_velocity_times_density", "closure.py",
     "u = np.stack([np.tensordot(Cf[:, a], g, axes=(0, 0)) for a in range(3)]) / rho",
     "u = np.stack([np.tensordot(Cf[:, a], g, axes=(0, 0)) for a in range(3)]) * rho", [CL]),
    ("features_shear_components_swapped", "closure.py",
     "pxy, pxz, pyz = P[0, 1] / s, P[0, 2] / s, P[1, 2] / s",
     "pxy, pxz, pyz = P[0, 2] / s, P[0, 1] / s, P[1, 2] / s", [CL]),
    ("features_third_order_scale", "closure.py",
     "q.append(np.tensordot(w, d, axes=(0, 0)) / s)", "q.append(np.tensordot(w, d, axes=(0, 0)))", [CL]),
    ("closure_step_features_of_the_old_state", "closure.py",
     "d_tau, _ = forward(theta, features(g[:, fluid], tau))",
     "d_tau, _ = forward(theta, features(f[:, fluid], tau))", [CL]),
    ("backprop_through_wrong_layer", "closure.py",
     'dh1 = dz2 @ p["W2"]', 'dh1 = dz2 @ p["W2"].T', [CL]),
    ("adam_step_counter_frozen", "closure.py",
     "theta, m, v = adam(theta, g, m, v, k, lr=lr)", "theta, m, v = adam(theta, g, m, v, 1, lr=lr)", [CL]),
    ("fold_output_offset_sign", "closure.py",
     'p["b3"] = p["b3"] * y_sd + y_mean', 'p["b3"] = p["b3"] * y_sd - y_mean', [CL]),
    ("loss_summed", "closure.py", "loss = float(np.mean(r * r))", "loss = float(np.sum(r * r))", [CL]),
    ("velocity_node_value_components", "lbm.py",
     "u = bc_node[0:3].copy()", "u = bc_node[1:4].copy()", [PINS]),
    ("taylor_green_closed_form_rate", "lbm.py",
     "return float(np.exp(-4.0 * nu * k * k * t))", "return float(np.exp(-2.0 * nu * k * k * t))", [PINS]),
    ("poiseuille_closed_form_factor", "lbm.py",
     "return g / (2.0 * nu) * (y + 0.5) * (h - 0.5 - y)", "return g / nu * (y + 0.5) * (h - 0.5 - y)",
     [PINS]),
    ("explosion_first_substep_two_hops", "multires.py",
     "                    ex = shift(c_up, c)\n", "                    ex = shift(c_up, c, 2)\n", [MR]),
    ("multires_closure_not_clamped", "multires.py",
     "tau[mine] = np.maximum(tau[mine] + d_tau, cl.TAU_MIN)", "tau[mine] = tau[mine] + d_tau", [MR]),
    ("partial_blocks_dropped", "layout.py",
     "nbz, nby, nbx = -(-nz // B), -(-ny // B), -(-nx // B)", "nbz, nby, nbx = nz // B, ny // B, nx // B",
     [PINS]),
    ("interface_blocks_not_first", "layout.py",
     "rows.sort(key=lambda r: r[0])", "rows.sort(key=lambda r: r[0][1])", [PINS]),
    ("conservation_momentum_axis", "lbm.py",
     "j = [float(np.tensordot(Cf[:, a], f, axes=(0, 0)).sum()) for a in range(3)]",
     "j = [float(np.tensordot(Cf[:, 0], f, axes=(0, 0)).sum()) for a in range(3)]", [PINS]),
    ("minibatch_modulus", "closure.py",
     "return np.array([splitmix64(seed + c0 + b) % n for b in range(batch)]",
     "return np.array([splitmix64(seed + c0 + b) % (n - 1) for b in range(batch)]", [CL]),
    ("morton_z_bit_misplaced", "layout.py",
     "code |= ((bz >> k) & 1) << (3 * k + 2)", "code |= ((bz >> k) & 1) << (3 * k + 1)", [PINS]),
    ("bc_index_rank_not_advanced", "layout.py",
     "                        rank += 1\n", "                        rank += 0\n", [PINS]),
    ("parameter_layout_b2_w3_swapped", "closure.py",
     '("b2", (HIDDEN,)), ("W3", (HIDDEN,))', '("W3", (HIDDEN,)), ("b2", (HIDDEN,))', [CL]),
    ("multires_shift_axes_swapped", "multires.py",
     "return np.roll(a, shift=(k * int(c[2]), k * int(c[1]), k * int(c[0])), axis=(-3, -2, -1))",
     "return np.roll(a, shift=(k * int(c[0]), k * int(c[1]), k * int(c[2])), axis=(-3, -2, -1))", [MR]),
    ("single_resolution_shift_axes_swapped", "lbm.py",
     "return np.roll(a, shift=(cz, cy, cx), axis=(0, 1, 2))",
     "return np.roll(a, shift=(cx, cy, cz), axis=(0, 1, 2))", [PINS]),
    ("level_owner_lookup_axes_swapped", "layout.py",
     "owner = own[lv][q[2] * B, q[1] * B, q[0] * B]", "owner = own[lv][q[0] * B, q[1] * B, q[2] * B]",
     [PINS, MR]),
    ("fine_octant_bits_swapped", "layout.py",
     "f = (2 * q[0] + (j & 1), 2 * q[1] + ((j >> 1) & 1), 2 * q[2] + (j >> 2))",
     "f = (2 * q[0] + (j >> 2), 2 * q[1] + ((j >> 1) & 1), 2 * q[2] + (j & 1))", [PINS, MR]),
]


def _copy_tree(dst, oracle_file=None, old=None, new=None):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    pkg = os.path.join(dst, "paper_2503_07898_gb300")
    os.makedirs(pkg)
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_2503_07898_gb300", f), pkg)
    tdir = os.path.join(dst, "tests")
    os.makedirs(tdir)
    for f in ("conftest.py", PINS, Q27, MR, CL):
        shutil.copy(os.path.join(ROOT, "tests", f), tdir)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), dst)
    if oracle_file is not None:
        path = os.path.join(dst, "oracle", oracle_file)
        src = open(path).read()
        assert src.count(old) == 1, f"planted edit must match exactly once in {oracle_file}: {old!r}"
        open(path, "w").write(src.replace(old, new))


def _run_pins(dst, files):
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    env.update(PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"]
    cmd += [os.path.join("tests", f) for f in files]
    r = subprocess.run(cmd, cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def _case(m):
    name, ofile, old, new, files = m
    with tempfile.TemporaryDirectory(prefix="oracle_mut_") as d:
        _copy_tree(d, ofile, old, new)
        return _run_pins(d, files)


UNMODIFIED = ("unmodified", None, None, None, [PINS, Q27, MR, CL])


@pytest.fixture(scope="module")
def outcomes():
    """Run the unmodified copy and every planted mistake once, in parallel
    interpreters."""
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {m[0]: ex.submit(_case, m) for m in [UNMODIFIED] + MUTATIONS}
        return {k: f.result() for k, f in futs.items()}


def test_unmodified_copy_passes_the_pins(outcomes):
    rc, out = outcomes["unmodified"]
    assert rc == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, out = outcomes[name]
    # 1: tests ran and some failed; anything else (collection error, crash)
    # would not show that a pin caught the mistake
    assert rc == 1, f"{name}: pytest exit code {rc}\n{out}"
