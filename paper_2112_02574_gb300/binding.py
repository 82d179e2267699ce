"""Thin Python binding of the C ABI in include/sc.h (argument marshalling only).

Every function named ``sc_*`` here calls the C entry point of the same name in
libscgb.so; PyTorch provides device memory and streams.  There is no fallback:
if the library is missing, importing this module raises ImportError.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libscgb.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sc.h")

SC_OK, SC_EINVAL, SC_ENOMEM, SC_ECUDA, SC_ENAN, SC_ETIMEOUT, SC_EUNSUPPORTED = range(7)
SC_D2Q9, SC_D3Q19 = 0, 1
SC_FORCE_E4, SC_FORCE_E6 = 0, 1
SC_PSI_N, SC_PSI_EXP = 0, 1
SC_STORE_F32, SC_STORE_F16, SC_STORE_BF16, SC_STORE_F64 = 0, 1, 2, 3
SC_PROFILE_RADIAL, SC_PROFILE_PLANAR_Z, SC_PROFILE_AXIS_X = 0, 1, 2
STATUS_NAMES = {0: "SC_OK", 1: "SC_EINVAL", 2: "SC_ENOMEM", 3: "SC_ECUDA", 4: "SC_ENAN", 5: "SC_ETIMEOUT",
                6: "SC_EUNSUPPORTED"}


class ScError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class sc_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("lattice", ctypes.c_int32), ("stencil", ctypes.c_int32), ("psi_self", ctypes.c_int32),
        ("storage", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("tile_z", ctypes.c_int32),
        ("variant", ctypes.c_int32), ("stages", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
        ("tau", ctypes.c_double * 2), ("G", ctypes.c_double), ("G_self", ctypes.c_double * 2),
    ]


def make_params(shape, lattice=SC_D3Q19, stencil=SC_FORCE_E4, psi_self=SC_PSI_EXP, storage=SC_STORE_F32,
                tau=(1.0, 1.0), G=0.0, G_self=(0.0, 0.0), tile_y=0, tile_z=0, variant=0, stages=0,
                blocks_per_sm=0) -> sc_params:
    """sc_params for a lattice of shape (nx, ny, nz); variant 0 auto, 1 generic, 2 staged step
    kernel; stages / blocks_per_sm tune the staged kernel (0 = library default)."""
    nx, ny, nz = shape
    return sc_params(int(nx), int(ny), int(nz), int(lattice), int(stencil), int(psi_self), int(storage),
                     int(tile_y), int(tile_z), int(variant), int(stages), int(blocks_per_sm),
                     (ctypes.c_double * 2)(*tau), float(G), (ctypes.c_double * 2)(*G_self))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    P, V, D, I64 = ctypes.POINTER(sc_params), ctypes.c_void_p, ctypes.c_double, ctypes.c_int64
    I32, Z = ctypes.c_int32, ctypes.c_size_t
    sig = {
        "sc_workspace_bytes": (Z, [P]),
        "sc_create": (I32, [P, V, V, V, Z, V, ctypes.POINTER(V)]),
        "sc_step": (I32, [V, I64]),
        "sc_moments": (I32, [V, V, V, V]),
        "sc_get_populations": (I32, [V, V]),
        "sc_set_populations": (I32, [V, V]),
        "sc_state_bytes": (Z, [V]),
        "sc_get_state": (I32, [V, V, Z]),
        "sc_set_state": (I32, [V, V, Z]),
        "sc_pressure_profile": (I32, [V, I32, ctypes.POINTER(D), D, I32, V]),
        "sc_bulk_pressure_at": (I32, [V, ctypes.POINTER(I32), V]),
        "sc_sigma_minimum": (I32, [V, I32, V, I32, D, D, D, V, V]),
        "sc_sigma0_flat": (I32, [V, I32, V, V]),
        "sc_curvature_fit": (I32, [V, V, I32, I32, V, V, V]),
        "sc_pressure_profile_noalloc": (I32, [P, V, V, I32, ctypes.POINTER(D), D, I32, V, V]),
        "sc_totals": (I32, [V, V]),
        "sc_sync": (I32, [V]),
        "sc_run_host": (I32, [P, V, V, I64, V, V, V, Z, V]),
        "sc_surface_of_tension": (I32, [V, I32, ctypes.POINTER(D), D, I32, D, D, D, V, V]),
        "sc_diagnostics": (I32, [V, V, I32, D, V]),
        "sc_run_host_sigma": (I32, [P, V, V, I64, ctypes.POINTER(D), D, I32, V, V, V, V, Z, V]),
        "sc_kernel_launches": (I64, [V]),
        "sc_step_config": (I32, [V, ctypes.POINTER(ctypes.c_int32), I32]),
        "sc_batch_workspace_bytes": (Z, [I32, P]),
        "sc_batch_create": (I32, [I32, P, ctypes.POINTER(V), ctypes.POINTER(V), V, Z, V, ctypes.POINTER(V)]),
        "sc_batch_step": (I32, [V, I64]),
        "sc_batch_member": (V, [V, I32]),
        "sc_batch_launches": (I64, [V]),
        "sc_batch_variant": (I32, [V]),
        "sc_batch_retire": (I32, [V, I32]),
        "sc_batch_active": (I32, [V]),
        "sc_batch_set_persistent": (I32, [V, I32]),
        "sc_selftest_wait_timeout": (I32, [V, I32]),
        "sc_velocity_change": (I32, [V, V, V]),
        "sc_centre_of_mass": (I32, [V, I32, D, V]),
        "sc_batch_destroy": (None, [V]),
        "sc_reference_density": (I32, [V, ctypes.POINTER(D)]),
        "sc_destroy": (None, [V]),
        "sc_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


def declared_symbols(header: str = HEADER):
    """Names of the functions include/sc.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sc_[a-z_0-9]+)\s*\(", text)))


def _check(status: int):
    if status != SC_OK:
        raise ScError(status, lib.sc_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    assert isinstance(t, torch.Tensor) and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ----------------------------------------------------------- C-ABI mirrors
def sc_workspace_bytes(params: sc_params) -> int:
    return lib.sc_workspace_bytes(ctypes.byref(params))


def sc_create(params, nA0, nB0, workspace, stream=None):
    ctx = ctypes.c_void_p()
    _check(lib.sc_create(ctypes.byref(params), _ptr(nA0), _ptr(nB0), _ptr(workspace), workspace.numel(),
                         _stream_ptr(stream), ctypes.byref(ctx)))
    return ctx


def sc_step(ctx, nsteps: int):
    _check(lib.sc_step(ctx, int(nsteps)))


def sc_moments(ctx, nA, nB, u=None):
    _check(lib.sc_moments(ctx, _ptr(nA), _ptr(nB), _ptr(u)))


def sc_get_populations(ctx, f):
    _check(lib.sc_get_populations(ctx, _ptr(f)))


def sc_set_populations(ctx, f):
    _check(lib.sc_set_populations(ctx, _ptr(f)))


def sc_state_bytes(ctx) -> int:
    return lib.sc_state_bytes(ctx)


def sc_get_state(ctx, dst):
    _check(lib.sc_get_state(ctx, _ptr(dst), dst.numel() * dst.element_size()))


def sc_set_state(ctx, src):
    _check(lib.sc_set_state(ctx, _ptr(src), src.numel() * src.element_size()))


def sc_pressure_profile(ctx, kind, centre, bin_width, nbins, out):
    c = (ctypes.c_double * 3)(*[float(v) for v in centre])
    _check(lib.sc_pressure_profile(ctx, int(kind), c, float(bin_width), int(nbins), _ptr(out)))


def sc_pressure_profile_noalloc(params, nA, nB, kind, centre, bin_width, nbins, out, stream=None):
    """Profile from device density fields with no device allocation (see include/sc.h)."""
    c = (ctypes.c_double * 3)(*[float(v) for v in centre])
    _check(lib.sc_pressure_profile_noalloc(ctypes.byref(params), _ptr(nA), _ptr(nB), int(kind), c,
                                           float(bin_width), int(nbins), _ptr(out), _stream_ptr(stream)))


def sc_bulk_pressure_at(ctx, node, out):
    n = (ctypes.c_int32 * 3)(*[int(v) for v in node])
    _check(lib.sc_bulk_pressure_at(ctx, n, _ptr(out)))


def sc_sigma_minimum(rows, P_in_out, dim, R_lo, R_hi, R_step, out, stream=None):
    _check(lib.sc_sigma_minimum(_ptr(rows), rows.shape[0], _ptr(P_in_out), int(dim), float(R_lo), float(R_hi),
                                float(R_step), _ptr(out), _stream_ptr(stream)))


def sc_surface_of_tension(ctx, kind, centre, bin_width, nbins, R_lo, R_hi, R_step, out, rows=None):
    c = None if centre is None else (ctypes.c_double * 3)(*[float(v) for v in centre])
    _check(lib.sc_surface_of_tension(ctx, int(kind), c, float(bin_width), int(nbins), float(R_lo), float(R_hi),
                                     float(R_step), _ptr(out), _ptr(rows)))


def sc_diagnostics(ctx, u_prev, component, background, out):
    _check(lib.sc_diagnostics(ctx, _ptr(u_prev), int(component), float(background), _ptr(out)))


def sc_run_host_sigma(params, nA0, nB0, nsteps, centre, bin_width, nbins, nA, nB, result, workspace, stream=None):
    """Host tensors in and out (result: host float64 [8]); see include/sc.h."""
    c = None if centre is None else (ctypes.c_double * 3)(*[float(v) for v in centre])
    _check(lib.sc_run_host_sigma(ctypes.byref(params), _ptr(nA0), _ptr(nB0), int(nsteps), c, float(bin_width),
                                 int(nbins), _ptr(nA), _ptr(nB), _ptr(result), _ptr(workspace), workspace.numel(),
                                 _stream_ptr(stream)))


def sc_sigma0_flat(rows, out, stream=None):
    _check(lib.sc_sigma0_flat(_ptr(rows), rows.shape[0], _ptr(out), _stream_ptr(stream)))


def sc_curvature_fit(Rs, sigma_s, order, sigma0, out, stream=None):
    _check(lib.sc_curvature_fit(_ptr(Rs), _ptr(sigma_s), int(Rs.numel()), int(order),
                                _ptr(sigma0) if sigma0 is not None else None, _ptr(out), _stream_ptr(stream)))


def sc_totals(ctx, out):
    _check(lib.sc_totals(ctx, _ptr(out)))


def sc_sync(ctx):
    _check(lib.sc_sync(ctx))


def sc_selftest_wait_timeout(ctx, max_polls: int):
    _check(lib.sc_selftest_wait_timeout(ctx, int(max_polls)))


def sc_run_host(params, nA0, nB0, nsteps, nA, nB, workspace, stream=None):
    """Host-buffer entry point: nA0, nB0, nA, nB are CPU float64 tensors (pinned or not)."""
    for t in (nA0, nB0, nA, nB):
        assert t.device.type == "cpu" and t.dtype == torch.float64 and t.is_contiguous()
    _check(lib.sc_run_host(ctypes.byref(params), _ptr(nA0), _ptr(nB0), int(nsteps), _ptr(nA), _ptr(nB),
                           _ptr(workspace), workspace.numel(), _stream_ptr(stream)))


def sc_batch_workspace_bytes(params_list) -> int:
    arr = (sc_params * len(params_list))(*params_list)
    return lib.sc_batch_workspace_bytes(len(params_list), arr)


def sc_batch_create(params_list, nA0_list, nB0_list, workspace, stream=None):
    n = len(params_list)
    arr = (sc_params * n)(*params_list)
    a = (ctypes.c_void_p * n)(*[t.data_ptr() for t in nA0_list])
    b = (ctypes.c_void_p * n)(*[t.data_ptr() for t in nB0_list])
    out = ctypes.c_void_p()
    _check(lib.sc_batch_create(n, arr, a, b, _ptr(workspace), workspace.numel(), _stream_ptr(stream),
                               ctypes.byref(out)))
    return out


def sc_batch_step(batch, nsteps: int):
    _check(lib.sc_batch_step(batch, int(nsteps)))


def sc_batch_member(batch, k: int):
    ctx = lib.sc_batch_member(batch, int(k))
    if not ctx:
        raise ScError(SC_EINVAL, sc_last_error())
    return ctypes.c_void_p(ctx)


def sc_batch_launches(batch) -> int:
    return lib.sc_batch_launches(batch)


def sc_batch_variant(batch) -> int:
    return lib.sc_batch_variant(batch)


def sc_batch_retire(batch, k):
    _check(lib.sc_batch_retire(batch, int(k)))


def sc_batch_active(batch) -> int:
    return lib.sc_batch_active(batch)


def sc_batch_set_persistent(batch, on: bool):
    _check(lib.sc_batch_set_persistent(batch, int(bool(on))))


def sc_velocity_change(ctx, u_prev, out):
    _check(lib.sc_velocity_change(ctx, _ptr(u_prev), _ptr(out)))


def sc_centre_of_mass(ctx, component, background, out):
    _check(lib.sc_centre_of_mass(ctx, int(component), float(background), _ptr(out)))


def sc_batch_destroy(batch):
    lib.sc_batch_destroy(batch)


def sc_kernel_launches(ctx) -> int:
    return lib.sc_kernel_launches(ctx)


STEP_CONFIG_KEYS = ("variant", "tile_y", "tile_z", "stages", "blocks_per_sm", "blocks", "zsplit_k", "zsplit_rem")


def sc_step_config(ctx) -> dict:
    out = (ctypes.c_int32 * 8)()
    _check(lib.sc_step_config(ctx, out, 8))
    return dict(zip(STEP_CONFIG_KEYS, list(out)))


def sc_reference_density(ctx):
    out = (ctypes.c_double * 2)()
    _check(lib.sc_reference_density(ctx, out))
    return out[0], out[1]


def sc_destroy(ctx):
    lib.sc_destroy(ctx)


def sc_last_error() -> str:
    return lib.sc_last_error().decode()


# ----------------------------------------------------------- convenience
class Simulation:
    """A simulation context with a torch-allocated workspace.

    nA0, nB0: float64 initial densities (CPU arrays / tensors or CUDA tensors),
    shape [nz, ny, nx] or flat.  All results are CUDA float64 tensors."""

    def __init__(self, params: sc_params, nA0, nB0, device="cuda", stream=None):
        self.params = params
        self.shape = (params.nx, params.ny, params.nz)
        self.N = params.nx * params.ny * params.nz
        self.Q = 19 if params.lattice == SC_D3Q19 else 9
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ws = sc_workspace_bytes(params)
        if ws == 0:
            raise ScError(SC_EINVAL, sc_last_error())
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        a = torch.as_tensor(nA0, dtype=torch.float64).reshape(-1).to(self.device).contiguous()
        b = torch.as_tensor(nB0, dtype=torch.float64).reshape(-1).to(self.device).contiguous()
        torch.cuda.synchronize(self.device)
        self.ctx = sc_create(params, a, b, self.workspace, self.stream)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            sc_destroy(ctx)
            self.ctx = None

    def step(self, n: int = 1):
        sc_step(self.ctx, n)

    def sync(self):
        sc_sync(self.ctx)

    def moments(self, with_u: bool = True):
        nA = torch.empty(self.N, dtype=torch.float64, device=self.device)
        nB = torch.empty_like(nA)
        u = torch.empty(3 * self.N, dtype=torch.float64, device=self.device) if with_u else None
        sc_moments(self.ctx, nA, nB, u)
        return nA, nB, (u.view(3, self.N) if with_u else None)

    def populations(self):
        f = torch.empty(2 * self.Q * self.N, dtype=torch.float64, device=self.device)
        sc_get_populations(self.ctx, f)
        return f.view(2, self.Q, self.N)

    def set_populations(self, f):
        f = torch.as_tensor(f, dtype=torch.float64).reshape(-1).to(self.device).contiguous()
        sc_set_populations(self.ctx, f)

    def state(self):
        t = torch.empty(sc_state_bytes(self.ctx), dtype=torch.uint8, device=self.device)
        sc_get_state(self.ctx, t)
        return t

    def set_state(self, t):
        sc_set_state(self.ctx, t)

    def profile(self, kind, centre=(0.0, 0.0, 0.0), bin_width=0.5, nbins=1):
        out = torch.empty(nbins * 6, dtype=torch.float64, device=self.device)
        sc_pressure_profile(self.ctx, kind, centre, bin_width, nbins, out)
        return out.view(nbins, 6)

    def bulk_pressure(self, node):
        out = torch.empty(1, dtype=torch.float64, device=self.device)
        sc_bulk_pressure_at(self.ctx, node, out)
        return out

    def velocity_change(self, u_prev):
        """Section 4's velocity criterion since u_prev (CUDA float64 [3][N], updated in place):
        a CUDA tensor [1] with (1/N) sum_x sum_alpha |u_alpha - u_prev_alpha|."""
        out = torch.empty(1, dtype=torch.float64, device=self.device)
        sc_velocity_change(self.ctx, u_prev, out)
        return out

    def centre_of_mass(self, component: int, background: float):
        """(X, Y, Z, W) of component 0 (A) or 1 (B) counted above `background`: a CUDA tensor [4]."""
        out = torch.empty(4, dtype=torch.float64, device=self.device)
        sc_centre_of_mass(self.ctx, component, background, out)
        return out

    def totals(self):
        out = torch.empty(5, dtype=torch.float64, device=self.device)
        sc_totals(self.ctx, out)
        return out

    @property
    def launches(self) -> int:
        return sc_kernel_launches(self.ctx)

    @property
    def step_config(self) -> dict:
        """The step kernel this simulation launches (variant, tiles, split, blocks per launch)."""
        return sc_step_config(self.ctx)

    @property
    def nbar(self):
        return sc_reference_density(self.ctx)


class _Member(Simulation):
    """A batch member viewed as a Simulation (no own workspace; the batch owns the context)."""

    def __init__(self, batch, k, params, device):
        self.params = params
        self.shape = (params.nx, params.ny, params.nz)
        self.N = params.nx * params.ny * params.nz
        self.Q = 19 if params.lattice == SC_D3Q19 else 9
        self.device = device
        self.stream = batch.stream
        self._batch = batch  # keeps the batch (and its workspace) alive
        self.ctx = sc_batch_member(batch.handle, k)

    def __del__(self):
        pass  # the batch owns the context


class Batch:
    """Several lattices stepped together: one kernel launch per time step, or one
    persistent launch per 32 steps for a staged batch."""

    def __init__(self, params_list, fields, device="cuda", stream=None):
        self.params = list(params_list)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ws = sc_batch_workspace_bytes(self.params)
        if ws == 0:
            raise ScError(SC_EINVAL, sc_last_error())
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        a = [torch.as_tensor(f[0], dtype=torch.float64).reshape(-1).to(self.device).contiguous() for f in fields]
        b = [torch.as_tensor(f[1], dtype=torch.float64).reshape(-1).to(self.device).contiguous() for f in fields]
        torch.cuda.synchronize(self.device)
        self.handle = sc_batch_create(self.params, a, b, self.workspace, self.stream)
        self.members = [_Member(self, k, p, self.device) for k, p in enumerate(self.params)]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            sc_batch_destroy(h)
            self.handle = None

    def step(self, n: int = 1):
        sc_batch_step(self.handle, n)

    @property
    def launches(self) -> int:
        return sc_batch_launches(self.handle)

    @property
    def staged(self) -> bool:
        """True when the batch steps with the staged kernel."""
        return sc_batch_variant(self.handle) >= 2

    @property
    def persistent(self) -> bool:
        """True when 32-step runs go out as one persistent cooperative launch."""
        return sc_batch_variant(self.handle) == 3

    @persistent.setter
    def persistent(self, on: bool):
        sc_batch_set_persistent(self.handle, on)

    def retire(self, k: int):
        """Stop stepping member k (it keeps its state for analysis)."""
        sc_batch_retire(self.handle, k)

    @property
    def active(self) -> int:
        return sc_batch_active(self.handle)


def surface_of_tension(sim: Simulation, centre=None, bin_width=0.5, nbins=0, kind=SC_PROFILE_RADIAL, R_step=0.01):
    """sc_surface_of_tension on a simulation: returns (rows [nbins, 6], out[8]) as CUDA tensors,
    out = (dP, C, R_s, sigma_s, R_grid, sigma_grid, P_in, P_out); nbins 0 = the library default."""
    nx, ny, nz = sim.shape
    if not nbins:
        dim3 = sim.params.lattice == SC_D3Q19 and nz > 1
        half = nx if kind == SC_PROFILE_AXIS_X else (min(nx, ny, nz) if dim3 else min(nx, ny))
        nbins = half // 2 if kind == SC_PROFILE_AXIS_X else int(half / 2 / bin_width)
    rows = torch.empty((nbins, 6), dtype=torch.float64, device=sim.device)
    out = torch.empty(8, dtype=torch.float64, device=sim.device)
    sc_surface_of_tension(sim.ctx, kind, centre, bin_width, nbins, 0.0, 0.0, R_step, out, rows)
    return rows, out


def sigma0_flat(sim: Simulation):
    """sigma_0 of a periodic slab along z (section 4): planar profile, then
    sc_sigma0_flat, on the device.  Returns (rows, sigma_0 as a CUDA tensor [1])."""
    rows = sim.profile(SC_PROFILE_PLANAR_Z, (0.0, 0.0, 0.0), 1.0, sim.shape[2])
    out = torch.empty(1, dtype=torch.float64, device=sim.device)
    sc_sigma0_flat(rows, out, sim.stream)
    return rows, out


def curvature_fit(Rs, sigma_s, order=2, sigma0=None, stream=None):
    """Eq. sigma_c fit over droplets on the device: Rs, sigma_s CUDA float64
    tensors (R_s negative for droplets of the other component), sigma0 a CUDA
    float64 [1] tensor or None (fitted).  Returns out[4] = (sigma_0, delta,
    2kbar + k, rms residual)."""
    out = torch.empty(4, dtype=torch.float64, device=Rs.device)
    sc_curvature_fit(Rs.contiguous(), sigma_s.contiguous(), order, sigma0, out, stream)
    return out
