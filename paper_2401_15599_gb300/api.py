"""PyTorch-facing wrappers of the libtacaw C-ABI (argument marshalling only).

Tensors provide device memory and the current CUDA stream; every step of the
computation runs in the library's CUDA kernels.  Functions take a grid
object with attributes nx, ny, lx, ly, n_slices, dz, z0, kev, bandlimit.
"""

from __future__ import annotations

import ctypes

import torch

from . import _lib as L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _need_cuda(name, t, dtype, ndim=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions")


def _workspace(query, device):
    nbytes = ctypes.c_size_t(0)
    query(ctypes.c_void_p(0), ctypes.byref(nbytes))
    ws = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8, device=device)
    return ws, nbytes


def status(device=None):
    """Wait for the current stream, then raise TacawError (ETIMEOUT) if a bounded
    device wait of an earlier call gave up since the last status check (its
    outputs are incomplete); the flag is cleared by reading it."""
    dev = torch.device("cuda") if device is None else torch.device(device)
    L.check("tacaw_status", L.load().tacaw_status(_stream(dev)))


def set_wait_limit(polls):
    """Polls of the multislice row pass's bounded waits for calls enqueued from
    now on (0 gives up at once, for tests); None or a negative value restores
    the default."""
    L.check("tacaw_set_wait_limit", L.load().tacaw_set_wait_limit(-1 if polls is None else int(polls)))


def beam_constants(kev: float):
    lam, sig = ctypes.c_double(), ctypes.c_double()
    L.check("tacaw_beam_constants", L.load().tacaw_beam_constants(kev, ctypes.byref(lam), ctypes.byref(sig)))
    return lam.value, sig.value


def potential(grid, pos, species, amp_sigma, out=None, workspace=None):
    """Slice potentials V [T, n_slices, ny, nx] (float32, V*A) of positions pos [T, Na, 3]."""
    lib = L.load()
    _need_cuda("pos", pos, torch.float32, 3)
    _need_cuda("species", species, torch.int32, 1)
    n_t, n_atoms = pos.shape[0], pos.shape[1]
    if pos.shape[2] != 3 or species.shape[0] != n_atoms:
        raise ValueError("pos must be [T, Na, 3] and species [Na]")
    amp = torch.as_tensor(amp_sigma, dtype=torch.float32).reshape(-1, 2).contiguous().cpu()
    n_species = amp.shape[0]
    amp_c = (ctypes.c_float * (2 * n_species))(*amp.flatten().tolist())
    g = L.make_grid(grid)
    if out is None:
        out = torch.empty((n_t, grid.n_slices, grid.ny, grid.nx), dtype=torch.float32, device=pos.device)
    _need_cuda("out", out, torch.float32, 4)

    def call(ws, nbytes):
        return lib.tacaw_potential(ctypes.byref(g), n_t, n_atoms, _ptr(pos), _ptr(species), n_species,
                                   amp_c, _ptr(out), ws, nbytes, _stream(pos.device))

    nbytes = ctypes.c_size_t(0)
    L.check("tacaw_potential", call(ctypes.c_void_p(0), ctypes.byref(nbytes)))
    if workspace is None or workspace.numel() < nbytes.value:
        workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=pos.device)
    nbytes = ctypes.c_size_t(workspace.numel())
    L.check("tacaw_potential", call(_ptr(workspace), ctypes.byref(nbytes)))
    return out


def multislice(grid, V, psi_in=None, out=None, psi_sum=None, workspace=None, ms_flags=0):
    """Exit waves psi_q [T, ny, nx] (complex64, q-space, FFT order) for potentials V.
    ms_flags: tacaw_multislice flags choosing variants of the passes (TACAW_MS_WARP_ROWS,
    TACAW_MS_BLOCK_COLS, or TACAW_MS_QUEUE alone; the tuner picks them per grid and GPU)."""
    lib = L.load()
    _need_cuda("V", V, torch.float32, 4)
    n_t = V.shape[0]
    if tuple(V.shape[1:]) != (grid.n_slices, grid.ny, grid.nx):
        raise ValueError("V must be [T, n_slices, ny, nx]")
    if out is None:
        out = torch.empty((n_t, grid.ny, grid.nx), dtype=torch.complex64, device=V.device)
    _need_cuda("out", out, torch.complex64, 3)
    if psi_in is not None:
        _need_cuda("psi_in", psi_in, torch.complex64, 2)
    if psi_sum is not None:
        _need_cuda("psi_sum", psi_sum, torch.complex128)
    g = L.make_grid(grid)

    def call(ws, nbytes):
        return lib.tacaw_multislice(ctypes.byref(g), n_t, _ptr(V), _ptr(psi_in), _ptr(out), _ptr(psi_sum),
                                    int(ms_flags), ws, nbytes, _stream(V.device))

    nbytes = ctypes.c_size_t(0)
    L.check("tacaw_multislice", call(ctypes.c_void_p(0), ctypes.byref(nbytes)))
    if workspace is None or workspace.numel() < nbytes.value:
        workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=V.device)
    nbytes = ctypes.c_size_t(workspace.numel())
    L.check("tacaw_multislice", call(_ptr(workspace), ctypes.byref(nbytes)))
    return out


_PRECISION = {"fp32": L.TACAW_FP32, "bf16x3": L.TACAW_BF16X3, "fft32": L.TACAW_FFT32, "bf16x6": L.TACAW_BF16X6}


def spectrum(psi, dt_fs, omega_meV=None, psi_sum=None, precision="fp32", kubo=False,
             temperature_K=300.0, normalize=False, out=None, i_el=None, workspace=None):
    """I(q, E) [nq, n_omega] (float32) and I_el [nq] (float64) from psi [T, nq] (complex64)."""
    lib = L.load()
    if psi.dim() > 2:
        psi = psi.reshape(psi.shape[0], -1)
    _need_cuda("psi", psi, torch.complex64, 2)
    n_t, nq = psi.shape
    dev = psi.device
    if omega_meV is not None:
        omega_meV = torch.as_tensor(omega_meV, dtype=torch.float64).to(dev).contiguous()
        n_w = omega_meV.numel()
    else:
        n_w = n_t
    if psi_sum is not None:
        _need_cuda("psi_sum", psi_sum, torch.complex128)
    if out is None:
        out = torch.empty((nq, n_w), dtype=torch.float32, device=dev)
    if i_el is None:
        i_el = torch.empty(nq, dtype=torch.float64, device=dev)
    _need_cuda("out", out, torch.float32, 2)
    _need_cuda("i_el", i_el, torch.float64, 1)
    flags = (L.TACAW_KUBO if kubo else 0) | (L.TACAW_NORMALIZE if normalize else 0)
    prec = _PRECISION[precision]

    def call(ws, nbytes):
        return lib.tacaw_spectrum(nq, n_t, float(dt_fs), n_w, _ptr(omega_meV), _ptr(psi), _ptr(psi_sum),
                                  _ptr(out), _ptr(i_el), prec, flags, float(temperature_K), ws, nbytes,
                                  _stream(dev))

    nbytes = ctypes.c_size_t(0)
    L.check("tacaw_spectrum", call(ctypes.c_void_p(0), ctypes.byref(nbytes)))
    if workspace is None or workspace.numel() < nbytes.value:
        workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
    nbytes = ctypes.c_size_t(workspace.numel())
    L.check("tacaw_spectrum", call(_ptr(workspace), ctypes.byref(nbytes)))
    return out, i_el


def _call_with_workspace(fn_name, call, device, workspace=None):
    nbytes = ctypes.c_size_t(0)
    L.check(fn_name, call(ctypes.c_void_p(0), ctypes.byref(nbytes)))
    if workspace is None or workspace.numel() < nbytes.value:
        workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=device)
    nbytes = ctypes.c_size_t(workspace.numel())
    L.check(fn_name, call(_ptr(workspace), ctypes.byref(nbytes)))


def spectrum_segments(psi, dt_fs, seg_len, hop, n_sets=0, omega_meV=None, precision="fp32", kubo=False,
                      temperature_K=300.0, normalize=False, out=None, i_el=None, workspace=None):
    """I(q, E) [nq, n_omega] (float32) and I_el [nq] (float64) averaged over sets of
    seg_len consecutive snapshots of psi [T, nq] offset by hop (n_sets = 0: all sets)."""
    lib = L.load()
    if psi.dim() > 2:
        psi = psi.reshape(psi.shape[0], -1)
    _need_cuda("psi", psi, torch.complex64, 2)
    n_t, nq = psi.shape
    dev = psi.device
    if omega_meV is not None:
        omega_meV = torch.as_tensor(omega_meV, dtype=torch.float64).to(dev).contiguous()
    n_w = seg_len if omega_meV is None else omega_meV.numel()
    if out is None:
        out = torch.empty((nq, n_w), dtype=torch.float32, device=dev)
    if i_el is None:
        i_el = torch.empty(nq, dtype=torch.float64, device=dev)
    _need_cuda("out", out, torch.float32, 2)
    _need_cuda("i_el", i_el, torch.float64, 1)
    flags = (L.TACAW_KUBO if kubo else 0) | (L.TACAW_NORMALIZE if normalize else 0)
    prec = _PRECISION[precision]

    def call(ws, nbytes):
        return lib.tacaw_spectrum_segments(nq, n_t, float(dt_fs), int(seg_len), int(hop), int(n_sets), n_w,
                                           _ptr(omega_meV), _ptr(psi), _ptr(out), _ptr(i_el), prec, flags,
                                           float(temperature_K), ws, nbytes, _stream(dev))
    _call_with_workspace("tacaw_spectrum_segments", call, dev, workspace)
    return out, i_el


def qep_intensity(psi, t0=0, stride=1, n=0, out=None):
    """(1/n) sum_j |psi(q, t0 + j stride)|^2 [nq] (float64) from psi [T, nq] (complex64)."""
    lib = L.load()
    if psi.dim() > 2:
        psi = psi.reshape(psi.shape[0], -1)
    _need_cuda("psi", psi, torch.complex64, 2)
    n_t, nq = psi.shape
    if out is None:
        out = torch.empty(nq, dtype=torch.float64, device=psi.device)
    _need_cuda("out", out, torch.float64, 1)
    L.check("tacaw_qep_intensity", lib.tacaw_qep_intensity(nq, n_t, int(t0), int(stride), int(n), _ptr(psi),
                                                           _ptr(out), _stream(psi.device)))
    return out


def energy_integral(inten, i_el=None, out=None):
    """I_el[q] + sum_k I[q, k] [nq] (float64) from I [nq, n_omega] (float32)."""
    lib = L.load()
    _need_cuda("I", inten, torch.float32, 2)
    nq, n_w = inten.shape
    if i_el is not None:
        _need_cuda("i_el", i_el, torch.float64, 1)
    if out is None:
        out = torch.empty(nq, dtype=torch.float64, device=inten.device)
    _need_cuda("out", out, torch.float64, 1)
    L.check("tacaw_energy_integral", lib.tacaw_energy_integral(nq, n_w, _ptr(inten), _ptr(i_el), _ptr(out),
                                                               _stream(inten.device)))
    return out


def line_profile(values, lx, lambda_A):
    """Profile of values [ny, nx] (float64, FFT order) along k_y = 0 in ascending
    theta_x = lambda q_x: returns (line [nx], theta_x [nx] in mrad)."""
    lib = L.load()
    _need_cuda("values", values, torch.float64, 2)
    ny, nx = values.shape
    line = torch.empty(nx, dtype=torch.float64, device=values.device)
    theta = torch.empty(nx, dtype=torch.float64, device=values.device)
    L.check("tacaw_line_profile", lib.tacaw_line_profile(nx, ny, float(lx), float(lambda_A), _ptr(values),
                                                         _ptr(line), _ptr(theta), _stream(values.device)))
    return line, theta


def azimuthal_profile(values, lx, ly, lambda_A, dtheta_mrad, n_bins, workspace=None):
    """Mean of values [ny, nx] (float64, FFT order) in bins of theta = lambda |q|
    (mrad): returns (profile [n_bins] float64, counts [n_bins] int32)."""
    lib = L.load()
    _need_cuda("values", values, torch.float64, 2)
    ny, nx = values.shape
    dev = values.device
    prof = torch.empty(int(n_bins), dtype=torch.float64, device=dev)
    counts = torch.empty(int(n_bins), dtype=torch.int32, device=dev)

    def call(ws, nbytes):
        return lib.tacaw_azimuthal_profile(nx, ny, float(lx), float(ly), float(lambda_A), float(dtheta_mrad),
                                           int(n_bins), _ptr(values), _ptr(prof), _ptr(counts), ws, nbytes,
                                           _stream(dev))
    _call_with_workspace("tacaw_azimuthal_profile", call, dev, workspace)
    return prof, counts


def relative_difference(a, b, out=None):
    """(a - b) / (a + b) elementwise (0 where a + b = 0), float64 tensors of equal size."""
    lib = L.load()
    _need_cuda("a", a, torch.float64)
    _need_cuda("b", b, torch.float64)
    if a.numel() != b.numel():
        raise ValueError("a and b must have the same size")
    if out is None:
        out = torch.empty_like(a)
    _need_cuda("out", out, torch.float64)
    L.check("tacaw_relative_difference", lib.tacaw_relative_difference(a.numel(), _ptr(a), _ptr(b), _ptr(out),
                                                                       _stream(a.device)))
    return out


def probe(grid, alpha_mrad, defocus_A=0.0, x0=0.0, y0=0.0, device="cuda", out=None, workspace=None):
    """Convergent-probe incident wave [ny, nx] (complex64, real space) on the
    grid's box at its beam energy, for multislice(..., psi_in=...)."""
    lib = L.load()
    dev = torch.device(device) if out is None else out.device
    if out is None:
        out = torch.empty((int(grid.ny), int(grid.nx)), dtype=torch.complex64, device=dev)
    _need_cuda("out", out, torch.complex64, 2)

    def call(ws, nbytes):
        return lib.tacaw_probe(int(grid.nx), int(grid.ny), float(grid.lx), float(grid.ly), float(grid.kev),
                               float(alpha_mrad), float(defocus_A), float(x0), float(y0), _ptr(out), ws, nbytes,
                               _stream(dev))
    _call_with_workspace("tacaw_probe", call, dev, workspace)
    return out


def spectrum_backward(psi, dt_fs, dl_di, omega_meV=None, psi_sum=None, out=None, workspace=None):
    """dL/dpsi [T, nq] (complex64) given dL/dI [nq, n_omega] (float32), FP32."""
    lib = L.load()
    if psi.dim() > 2:
        psi = psi.reshape(psi.shape[0], -1)
    _need_cuda("psi", psi, torch.complex64, 2)
    _need_cuda("dl_di", dl_di, torch.float32, 2)
    n_t, nq = psi.shape
    dev = psi.device
    if omega_meV is not None:
        omega_meV = torch.as_tensor(omega_meV, dtype=torch.float64).to(dev).contiguous()
    n_w = n_t if omega_meV is None else omega_meV.numel()
    if tuple(dl_di.shape) != (nq, n_w):
        raise ValueError("dl_di must be [nq, n_omega]")
    if out is None:
        out = torch.empty((n_t, nq), dtype=torch.complex64, device=dev)
    _need_cuda("out", out, torch.complex64)

    def call(ws, nbytes):
        return lib.tacaw_spectrum_backward(nq, n_t, float(dt_fs), n_w, _ptr(omega_meV), _ptr(psi), _ptr(psi_sum),
                                           _ptr(dl_di), _ptr(out), ws, nbytes, _stream(dev))
    _call_with_workspace("tacaw_spectrum_backward", call, dev, workspace)
    return out


def multislice_backward(grid, V, dl_dpsi_q, psi_in=None, ckpt_every=0, out=None, workspace=None):
    """dL/dV [T, n_slices, ny, nx] (float32) given dL/d(exit waves) [T, ny, nx] (complex64)."""
    lib = L.load()
    _need_cuda("V", V, torch.float32, 4)
    _need_cuda("dl_dpsi_q", dl_dpsi_q, torch.complex64, 3)
    n_t = V.shape[0]
    if out is None:
        out = torch.empty_like(V)
    _need_cuda("out", out, torch.float32, 4)
    g = L.make_grid(grid)

    def call(ws, nbytes):
        return lib.tacaw_multislice_backward(ctypes.byref(g), n_t, _ptr(V), _ptr(psi_in), _ptr(dl_dpsi_q),
                                             _ptr(out), int(ckpt_every), ws, nbytes, _stream(V.device))
    _call_with_workspace("tacaw_multislice_backward", call, V.device, workspace)
    return out


def potential_backward(grid, pos, species, amp_sigma, dl_dv, out=None, workspace=None):
    """dL/d(amp, sigma) [n_species, 2] (float64, device) given dL/dV [T, n_slices, ny, nx]."""
    lib = L.load()
    _need_cuda("pos", pos, torch.float32, 3)
    _need_cuda("species", species, torch.int32, 1)
    _need_cuda("dl_dv", dl_dv, torch.float32, 4)
    n_t, n_atoms = pos.shape[0], pos.shape[1]
    amp = torch.as_tensor(amp_sigma, dtype=torch.float32).detach().reshape(-1, 2).contiguous().cpu()
    n_species = amp.shape[0]
    amp_c = (ctypes.c_float * (2 * n_species))(*amp.flatten().tolist())
    if out is None:
        out = torch.empty((n_species, 2), dtype=torch.float64, device=pos.device)
    g = L.make_grid(grid)

    def call(ws, nbytes):
        return lib.tacaw_potential_backward(ctypes.byref(g), n_t, n_atoms, _ptr(pos), _ptr(species), n_species,
                                            amp_c, _ptr(dl_dv), _ptr(out), ws, nbytes, _stream(pos.device))
    _call_with_workspace("tacaw_potential_backward", call, pos.device, workspace)
    return out


def multislice_batch(jobs, workspace=None, queue=False, wave=0, span=0):
    """Run several multislice jobs of uneven size in one call.

    jobs: sequence of dicts with keys grid, V [T, n_s, ny, nx] float32, out
    [T, ny, nx] complex64 and optionally psi_in [ny, nx] complex64 and
    psi_sum [ny, nx] complex128.  All tensors on the same CUDA device.
    queue: use tacaw_multislice_queue (square grids; one persistent launch per
    grid size over a device work queue, waves of `wave` snapshots and items of
    `span` rows or columns, 0 = defaults) instead of tacaw_multislice_batch (two
    launches per slice).
    """
    lib = L.load()
    arr = (L.TacawJob * max(1, len(jobs)))()
    dev = None
    for i, j in enumerate(jobs):
        V, out = j["V"], j["out"]
        _need_cuda("V", V, torch.float32, 4)
        _need_cuda("out", out, torch.complex64, 3)
        g = j["grid"]
        if tuple(V.shape[1:]) != (g.n_slices, g.ny, g.nx) or tuple(out.shape) != (V.shape[0], g.ny, g.nx):
            raise ValueError(f"job {i}: V must be [T, n_slices, ny, nx] and out [T, ny, nx]")
        psi_in, psi_sum = j.get("psi_in"), j.get("psi_sum")
        if psi_in is not None:
            _need_cuda("psi_in", psi_in, torch.complex64, 2)
        if psi_sum is not None:
            _need_cuda("psi_sum", psi_sum, torch.complex128)
        arr[i] = L.TacawJob(L.make_grid(g), int(V.shape[0]), V.data_ptr(),
                            psi_in.data_ptr() if psi_in is not None else None, out.data_ptr(),
                            psi_sum.data_ptr() if psi_sum is not None else None)
        dev = V.device
    if dev is None:
        return

    if queue:
        def call(ws, nbytes):
            return lib.tacaw_multislice_queue(arr, len(jobs), int(wave), int(span), ws, nbytes, _stream(dev))
        _call_with_workspace("tacaw_multislice_queue", call, dev, workspace)
        return

    def call(ws, nbytes):
        return lib.tacaw_multislice_batch(arr, len(jobs), ws, nbytes, _stream(dev))
    _call_with_workspace("tacaw_multislice_batch", call, dev, workspace)


def time_mean(psi_sum, n, out=None):
    """mean [nq] (complex128) = psi_sum [nq] (complex128) / n, on the device."""
    lib = L.load()
    _need_cuda("psi_sum", psi_sum, torch.complex128)
    nq = psi_sum.numel()
    if out is None:
        out = torch.empty(nq, dtype=torch.complex128, device=psi_sum.device)
    _need_cuda("out", out, torch.complex128)
    L.check("tacaw_time_mean", lib.tacaw_time_mean(nq, int(n), _ptr(psi_sum), _ptr(out), _stream(psi_sum.device)))
    return out


def spectrum_accumulate(psi_chunk, t0, dt_fs, omega_meV, m_ref, phi, precision="bf16x6", workspace=None):
    """phi [nq, n_omega] (complex64, in/out) += the transform of the chunk
    psi_chunk [n_chunk, nq] (snapshots t0 ..) centred on m_ref [nq] (complex128)."""
    lib = L.load()
    if psi_chunk.dim() > 2:
        psi_chunk = psi_chunk.reshape(psi_chunk.shape[0], -1)
    _need_cuda("psi_chunk", psi_chunk, torch.complex64, 2)
    _need_cuda("m_ref", m_ref, torch.complex128)
    _need_cuda("phi", phi, torch.complex64, 2)
    n_chunk, nq = psi_chunk.shape
    dev = psi_chunk.device
    omega = torch.as_tensor(omega_meV, dtype=torch.float64).to(dev).contiguous()
    n_w = omega.numel()
    if tuple(phi.shape) != (nq, n_w) or m_ref.numel() != nq:
        raise ValueError("phi must be [nq, n_omega] and m_ref [nq]")
    prec = _PRECISION[precision]

    def call(ws, nbytes):
        return lib.tacaw_spectrum_accumulate(nq, int(t0), n_chunk, float(dt_fs), n_w, _ptr(omega), _ptr(psi_chunk),
                                             _ptr(m_ref), _ptr(phi), prec, ws, nbytes, _stream(dev))

    _call_with_workspace("tacaw_spectrum_accumulate", call, dev, workspace)
    return phi


def spectrum_finish(phi, n_t, dt_fs, omega_meV, m_ref, psi_sum, kubo=False, temperature_K=300.0,
                    normalize=False, out=None, i_el=None, workspace=None):
    """I [nq, n_omega] (float32) and I_el [nq] (float64) from the accumulated phi."""
    lib = L.load()
    _need_cuda("phi", phi, torch.complex64, 2)
    _need_cuda("m_ref", m_ref, torch.complex128)
    _need_cuda("psi_sum", psi_sum, torch.complex128)
    nq, n_w = phi.shape
    dev = phi.device
    omega = torch.as_tensor(omega_meV, dtype=torch.float64).to(dev).contiguous()
    if omega.numel() != n_w:
        raise ValueError("omega_meV must have n_omega entries")
    if out is None:
        out = torch.empty((nq, n_w), dtype=torch.float32, device=dev)
    if i_el is None:
        i_el = torch.empty(nq, dtype=torch.float64, device=dev)
    _need_cuda("out", out, torch.float32, 2)
    _need_cuda("i_el", i_el, torch.float64, 1)
    flags = (L.TACAW_KUBO if kubo else 0) | (L.TACAW_NORMALIZE if normalize else 0)

    def call(ws, nbytes):
        return lib.tacaw_spectrum_finish(nq, int(n_t), float(dt_fs), n_w, _ptr(omega), _ptr(phi), _ptr(m_ref),
                                         _ptr(psi_sum), _ptr(out), _ptr(i_el), flags, float(temperature_K), ws,
                                         nbytes, _stream(dev))

    _call_with_workspace("tacaw_spectrum_finish", call, dev, workspace)
    return out, i_el


def time_to_spectrum_host(grid, pos_host, species, amp_sigma, dt_fs, batch, ms_flags=0, precision="fft32",
                          kubo=False, temperature_K=300.0, normalize=False, out=None, out_el=None, workspace=None):
    """The whole path in one library call: positions pos_host [T, Na, 3]
    (float32, CPU; page-locked for overlapped copies) -> I [nq, T] and I_el
    [nq] in host memory (natural energy grid).  Outputs are valid once the
    current stream has reached the end of the call."""
    lib = L.load()
    if pos_host.device.type != "cpu" or pos_host.dtype != torch.float32 or not pos_host.is_contiguous():
        raise ValueError("pos_host must be a contiguous float32 CPU tensor")
    _need_cuda("species", species, torch.int32, 1)
    n_t, n_atoms = int(pos_host.shape[0]), int(pos_host.shape[1])
    nq = int(grid.nx) * int(grid.ny)
    if out is None:
        out = torch.empty((nq, n_t), dtype=torch.float32).pin_memory()
    if out_el is None:
        out_el = torch.empty(nq, dtype=torch.float64).pin_memory()
    if out.device.type != "cpu" or tuple(out.shape) != (nq, n_t) or out.dtype != torch.float32:
        raise ValueError("out must be a float32 CPU tensor [nq, T]")
    if out_el.device.type != "cpu" or out_el.numel() != nq or out_el.dtype != torch.float64:
        raise ValueError("out_el must be a float64 CPU tensor [nq]")
    amp = torch.as_tensor(amp_sigma, dtype=torch.float32).reshape(-1, 2).contiguous().cpu()
    amp_c = (ctypes.c_float * amp.numel())(*amp.flatten().tolist())
    g = L.make_grid(grid)
    flags = (L.TACAW_KUBO if kubo else 0) | (L.TACAW_NORMALIZE if normalize else 0)
    dev = species.device

    def call(ws, nbytes):
        return lib.tacaw_time_to_spectrum_host(ctypes.byref(g), n_t, n_atoms, ctypes.c_void_p(pos_host.data_ptr()),
                                               _ptr(species), amp.shape[0], amp_c, float(dt_fs), int(batch),
                                               int(ms_flags), _PRECISION[precision],
                                               flags, float(temperature_K), ctypes.c_void_p(out.data_ptr()),
                                               ctypes.c_void_p(out_el.data_ptr()), ws, nbytes, _stream(dev))

    _call_with_workspace("tacaw_time_to_spectrum_host", call, dev, workspace)
    return out, out_el


def time_to_spectrum_host_workspace(grid, n_t, n_atoms, batch, precision="fft32", device="cuda"):
    """A device workspace large enough for time_to_spectrum_host with these sizes."""
    lib = L.load()
    g = L.make_grid(grid)
    amp = (ctypes.c_float * 2)(1.0, 1.0)
    nbytes = ctypes.c_size_t(0)
    null = ctypes.c_void_p(0)
    L.check("tacaw_time_to_spectrum_host",
            lib.tacaw_time_to_spectrum_host(ctypes.byref(g), int(n_t), int(n_atoms), null, null, 1, amp, 1.0,
                                            int(batch), 0, _PRECISION[precision], 0, 300.0, null, null, null,
                                            ctypes.byref(nbytes), null))
    return torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8, device=device)
