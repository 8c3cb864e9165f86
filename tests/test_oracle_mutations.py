"""Plant plausible mistakes in the oracle (CPU only) and check a pin fails.

Each mutation replaces one oracle function with a subtly wrong version (a
dropped factor, a flipped sign, a wrong index or axis); the pins in
``test_oracle_pins`` must reject every one of them.
"""

import numpy as np
import pytest
from scipy.special import erf

import oracle
import oracle.tacaw_oracle as T
from tests import test_oracle_pins as P


def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(T, name, fn)
    monkeypatch.setattr(oracle, name, fn)


def _prop_variant(sign=-1.0, dz_scale=1.0, bl=True):
    def prop(g):
        qx, qy = T.spatial_frequencies(g)
        q2 = qx[None, :] ** 2 + qy[:, None] ** 2
        p = np.exp(sign * 1j * np.pi * T.wavelength(g.kev) * g.dz * dz_scale * q2)
        return p * T.bandlimit_mask(g) if bl else p
    return prop


def _ms_variant(trans_sign=1.0, last_prop=True):
    def ms(g, v, psi_in=None):
        sig = T.interaction_constant(g.kev)
        prop = T.propagator(g)
        psi = np.ones((g.ny, g.nx), complex) if psi_in is None else np.asarray(psi_in, complex)
        out = None
        for s in range(g.n_slices):
            chi = np.exp(trans_sign * 1j * sig * v[s]) * psi
            out = T.fft2_unitary(chi)
            if last_prop or s + 1 < g.n_slices:
                out = prop * out
            if s + 1 < g.n_slices:
                psi = T.ifft2_unitary(out)
        return out
    return ms


def _weights_variant(root2=True, open_ends=True):
    def w(z, sigma, g):
        n = g.n_slices
        edges = g.z0 + g.dz * np.arange(n + 1)
        scale = np.sqrt(2.0) * sigma if root2 else sigma
        cdf = 0.5 * erf((edges - z) / scale)
        if open_ends:
            cdf[0], cdf[n] = -0.5, 0.5
        return cdf[1:] - cdf[:-1]
    return w


def _pot_variant(width2=2.0, shift=0.0, swap=False):
    def pot(g, pos, species, amp_sigma):
        pos = np.asarray(pos, float)
        amp_sigma = np.asarray(amp_sigma, float).reshape(-1, 2)
        x = (np.arange(g.nx) + shift) * g.lx / g.nx
        y = (np.arange(g.ny) + shift) * g.ly / g.ny
        v = np.zeros((g.n_slices, g.ny, g.nx))
        for a in range(pos.shape[0]):
            amp, sig = amp_sigma[int(np.asarray(species)[a])]
            px, py = (pos[a, 1], pos[a, 0]) if swap else (pos[a, 0], pos[a, 1])
            ddx = np.mod(x - px + g.lx / 2, g.lx) - g.lx / 2
            ddy = np.mod(y - py + g.ly / 2, g.ly) - g.ly / 2
            r2 = ddx[None, :] ** 2 + ddy[:, None] ** 2
            inside = (np.abs(ddx)[None, :] <= 6 * sig) & (np.abs(ddy)[:, None] <= 6 * sig)
            prof = amp * np.exp(-r2 / (width2 * sig * sig)) * inside
            v += T.slice_weights(pos[a, 2], sig, g)[:, None, None] * prof[None]
        return v
    return pot


def _tt_variant(inverse=False, shift=True):
    def tt(a, dt_fs, omega_meV=None):
        a = np.asarray(a, complex)
        if omega_meV is None:
            f = np.fft.ifft(a, axis=0) * a.shape[0] if inverse else np.fft.fft(a, axis=0)
            return (np.fft.fftshift(f, axes=0) if shift else f).T.copy()
        t = np.arange(a.shape[0]) * dt_fs
        sgn = 1j if inverse else -1j
        return a.T @ np.exp(sgn * np.outer(t, omega_meV) / T.HBAR_MEV_FS)
    return tt


def _spectrum_variant(subtract=True, power=2, norm_el=True):
    def spec(psi, dt_fs, omega_meV=None, kubo=False, temperature_K=300.0, normalize=False):
        psi = np.asarray(psi, complex)
        n_t = psi.shape[0]
        psi = psi.reshape(n_t, -1)
        m = T.time_mean(psi)
        iel = np.abs(m) ** 2
        a = psi - m[None] if subtract else psi
        inten = np.abs(T.temporal_transform(a, dt_fs, omega_meV)) ** 2 / float(n_t) ** power
        e = T.natural_energies(n_t, dt_fs) if omega_meV is None else np.asarray(omega_meV)
        if kubo:
            inten = inten * T.kubo_factor(e, temperature_K)[None]
        if normalize:
            tot = inten.sum() + (iel.sum() if norm_el else 0.0)
            inten, iel = inten / tot, iel / tot
        return inten, iel, e
    return spec


def _kubo_wrong(e, temperature_K):
    be = np.asarray(e, float) / (T.KB_MEV_PER_K * temperature_K)
    out = np.ones_like(be)
    nz = be != 0
    out[nz] = be[nz] / (1.0 - np.exp(be[nz]))
    return out


def _bl_max(g):
    qx, qy = T.spatial_frequencies(g)
    q2 = qx[None, :] ** 2 + qy[:, None] ** 2
    qmax = g.bandlimit * max(g.nx / (2 * g.lx), g.ny / (2 * g.ly))
    return (q2 <= qmax * qmax).astype(float)


def _segments_variant(stride_is_length=False, divide=True, global_mean=False):
    def seg(psi, dt_fs, seg_len, hop, n_sets=None, omega_meV=None, kubo=False, temperature_K=300.0,
            normalize=False):
        psi = np.asarray(psi, complex).reshape(np.shape(psi)[0], -1)
        if stride_is_length:        # offset confused with the overlap seg_len - hop
            stride = seg_len - hop if seg_len > hop else seg_len
            starts = T.segment_starts(psi.shape[0], seg_len, stride)
        else:
            starts = T.segment_starts(psi.shape[0], seg_len, hop, n_sets)
        inten, iel = 0.0, 0.0
        for s0 in starts:
            part = psi[s0:s0 + seg_len]
            if global_mean:
                part = part - psi.mean(axis=0) + part.mean(axis=0)
            i_g, iel_g, e = T.spectrum(part, dt_fs, omega_meV)
            inten, iel = inten + i_g, iel + iel_g
        if divide:
            inten, iel = inten / len(starts), iel / len(starts)
        if kubo:
            inten = inten * T.kubo_factor(e, temperature_K)[None]
        if normalize:
            tot = inten.sum() + iel.sum()
            inten, iel = inten / tot, iel / tot
        return inten, iel, e
    return seg


def _line_unshifted(values, lx, lam):
    values = np.asarray(values, float)
    nx = values.shape[1]
    return values[0], lam * np.fft.fftfreq(nx, d=lx / nx) * 1000.0


def _azimuthal_rounded(values, lx, ly, lam, dtheta, n_bins):
    values = np.asarray(values, float)
    ny, nx = values.shape
    b = np.round(T.scattering_angles(nx, ny, lx, ly, lam) / dtheta).ravel()
    keep = b < n_bins
    counts = np.bincount(b[keep].astype(int), minlength=n_bins)
    sums = np.bincount(b[keep].astype(int), weights=values.ravel()[keep], minlength=n_bins)
    return np.where(counts > 0, sums / np.maximum(counts, 1), 0.0), counts


def _probe_variant(defocus_sign=1.0, shift_sign=1.0, norm_power=0.5):
    def probe(g, alpha_mrad, defocus_A=0.0, x0=0.0, y0=0.0):
        qx, qy = T.spatial_frequencies(g)
        lam = T.wavelength(g.kev)
        inside = lam * np.sqrt(qx[None, :] ** 2 + qy[:, None] ** 2) * 1000.0 <= alpha_mrad
        q2 = qx[None, :] ** 2 + qy[:, None] ** 2
        phase = (-defocus_sign * np.pi * lam * defocus_A * q2
                 - shift_sign * 2.0 * np.pi * (qx[None, :] * x0 + qy[:, None] * y0))
        psi_q = np.where(inside, np.exp(1j * phase), 0.0) / np.count_nonzero(inside) ** norm_power
        return T.ifft2_unitary(psi_q)
    return probe


MUTATIONS = {
    "fft_missing_1_over_N": ("fft2_unitary", lambda p: np.fft.fft2(p)),
    "ifft_with_1_over_N": ("ifft2_unitary", lambda p: np.fft.ifft2(p)),
    "propagator_sign": ("propagator", _prop_variant(sign=+1.0)),
    "propagator_half_dz": ("propagator", _prop_variant(dz_scale=0.5)),
    "propagator_no_bandlimit": ("propagator", _prop_variant(bl=False)),
    "bandlimit_max_nyquist": ("bandlimit_mask", _bl_max),
    "transmission_sign": ("multislice", _ms_variant(trans_sign=-1.0)),
    "no_last_propagation": ("multislice", _ms_variant(last_prop=False)),
    "weights_missing_root2": ("slice_weights", _weights_variant(root2=False)),
    "weights_closed_ends": ("slice_weights", _weights_variant(open_ends=False)),
    "gaussian_width": ("projected_potential", _pot_variant(width2=1.0)),
    "pixel_centre_shift": ("projected_potential", _pot_variant(shift=0.5)),
    "xy_swapped": ("projected_potential", _pot_variant(swap=True)),
    "time_transform_sign": ("temporal_transform", _tt_variant(inverse=True)),
    "time_transform_unshifted": ("temporal_transform", _tt_variant(shift=False)),
    "no_mean_subtraction": ("spectrum", _spectrum_variant(subtract=False)),
    "power_over_T": ("spectrum", _spectrum_variant(power=1)),
    "normalise_without_elastic": ("spectrum", _spectrum_variant(norm_el=False)),
    "kubo_sign": ("kubo_factor", _kubo_wrong),
    "sum_not_mean": ("time_mean", lambda psi: np.sum(np.asarray(psi, complex), axis=0)),
    "energy_hbar_for_h": ("natural_energies",
                          lambda n, dt: np.fft.fftshift(np.fft.fftfreq(n, d=dt)) * T.HBAR_MEV_FS),
    "sigma_without_gamma": ("interaction_constant",
                            lambda kev: 2 * np.pi * T.ME_KG * T.E_C * T.wavelength(kev) * 1e-10
                            / T.PLANCK_J_S ** 2 * 1e-10),
    "segments_offset_as_overlap": ("segment_spectrum", _segments_variant(stride_is_length=True)),
    "segments_summed_not_averaged": ("segment_spectrum", _segments_variant(divide=False)),
    "segments_global_mean": ("segment_spectrum", _segments_variant(global_mean=True)),
    "qep_ignores_stride": ("qep_intensity",
                           lambda psi, t0=0, stride=1, n=None: np.mean(np.abs(np.asarray(psi, complex)) ** 2, axis=0)),
    "line_profile_fft_order": ("line_profile", _line_unshifted),
    "azimuthal_rounded_bins": ("azimuthal_profile", _azimuthal_rounded),
    "relative_difference_over_b": ("relative_difference",
                                   lambda a, b: (np.asarray(a, float) - b) / np.where(np.asarray(b) != 0, b, 1.0)),
    "probe_defocus_sign": ("probe", _probe_variant(defocus_sign=-1.0)),
    "probe_shift_sign": ("probe", _probe_variant(shift_sign=-1.0)),
    "probe_norm_not_sqrt": ("probe", _probe_variant(norm_power=1.0)),
    "wavelength_nonrelativistic": ("wavelength",
                                   lambda kev: T.PLANCK_J_S / np.sqrt(2 * T.ME_KG * kev * 1e3 * T.E_C)
                                   * 1e10),
}

PINS = [
    lambda: P.test_beam_constants_textbook_values(),
    lambda: P.test_energy_limits_match_paper_footnotes(),
    lambda: P.test_energy_grid_resolution_and_order(),
    lambda: P.test_fft2_unitary_bruteforce(4, 6),
    lambda: P.test_temporal_transform_bruteforce(8),
    lambda: P.test_energy_sign_loss_is_positive(),
    lambda: P.test_slice_weights_quadrature_and_sum(),
    lambda: P.test_potential_window_equals_bruteforce(),
    lambda: P.test_potential_integral_sum_rule(),
    lambda: P.test_potential_fourier_transform_analytic(),
    lambda: P.test_free_space_gaussian_beam_closed_form((128, 96, 64.0, 60.0)),
    lambda: P.test_uniform_potential_is_a_global_phase(),
    lambda: P.test_weak_phase_single_slice_first_order(),
    lambda: P.test_norm_conserved_without_bandlimit_and_lost_outside_it(),
    lambda: P.test_bandlimit_disc_radius(),
    lambda: P.test_parseval_energy_integral_equals_qep(),
    lambda: P.test_wiener_khinchin(),
    lambda: P.test_elastic_bin_zero_and_static_lattice(),
    lambda: P.test_kubo_factor_detailed_balance(),
    lambda: P.test_normalisation_sums_to_one(),
    lambda: P.test_segment_sets_match_paper(),
    lambda: P.test_segment_spectrum_bruteforce(),
    lambda: P.test_segment_spectrum_parseval_over_tiling_sets(),
    lambda: P.test_qep_subset_of_the_si_trajectory(),
    lambda: P.test_energy_integral_equals_qep_of_all_snapshots(),
    lambda: P.test_line_profile_bragg_spots_of_a_static_crystal(),
    lambda: P.test_azimuthal_profile_bruteforce(),
    lambda: P.test_relative_difference_closed_forms(),
    lambda: P.test_probe_aperture_and_normalisation(),
    lambda: P.test_probe_position_is_a_circular_shift(),
    lambda: P.test_probe_defocus_is_free_propagation(),
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_some_pin_rejects_mutation(name, monkeypatch):
    target, fn = MUTATIONS[name]
    _patch(monkeypatch, target, fn)
    caught = []
    for i, pin in enumerate(PINS):
        try:
            pin()
        except AssertionError:     # a failed pin (not a crash of the mutant) rejects it
            caught.append(i)
    assert caught, f"no pin rejects the mutation {name}"
