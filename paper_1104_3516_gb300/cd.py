"""Python binding of the C ABI in ``include/cd_api.h`` (argument marshalling only).

Every compute step runs in the CUDA library ``_lib/libcd_gb300.so``; this
module only passes torch tensors' device pointers and the current CUDA stream.
There is no CPU fallback: if the library is missing the import of a system
fails with an error that says how to build it.

The functions ``cd_create_system`` ... ``cd_last_error`` mirror the C entry
points one to one; :class:`CDSystem` bundles them with the torch tensors that
own the particle state and the workspace.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcd_gb300.so")

CD_OK, CD_ERR_INVALID_ARG, CD_ERR_CUDA, CD_ERR_OOM, CD_ERR_CAPACITY, CD_ERR_NOT_CONVERGED, CD_ERR_TIMEOUT, \
    CD_ERR_STATE = range(8)
STATUS_NAMES = ["CD_OK", "CD_ERR_INVALID_ARG", "CD_ERR_CUDA", "CD_ERR_OOM", "CD_ERR_CAPACITY",
                "CD_ERR_NOT_CONVERGED", "CD_ERR_TIMEOUT", "CD_ERR_STATE"]
CD_FP64, CD_FP32 = 0, 1
CD_CONV_NONE, CD_CONV_GLOBAL_REL, CD_CONV_GLOBAL_SQ, CD_CONV_LOCAL = -1, 0, 1, 2


class CDError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {message}")
        self.status = status
        self.message = message


class cd_params(C.Structure):
    _fields_ = [
        ("dim", C.c_int64),
        ("precision", C.c_int64),
        ("dt", C.c_double),
        ("mu", C.c_double),
        ("gravity", C.c_double * 3),
        ("box_lo", C.c_double * 3),
        ("box_hi", C.c_double * 3),
        ("periodic", C.c_int64 * 3),
        ("wall_mask", C.c_int64),
        ("wall_pos", C.c_double * 6),
        ("wall_vel", C.c_double * 18),
        ("delta", C.c_double),
        ("alpha", C.c_double),
        ("criterion", C.c_int64),
        ("max_sweeps", C.c_int64),
        ("warm_start", C.c_int64),
        ("rotations", C.c_int64),
        ("seed", C.c_uint64),
        ("max_contacts", C.c_int64),
        ("timing", C.c_int64),
        ("parallel_p", C.c_double),
        ("tape_steps", C.c_int64),
        ("adjoint_compliance", C.c_double),
        ("use_graph", C.c_int64),
        ("sweep_threads", C.c_int64),
        ("sweep_blocks_per_sm", C.c_int64),
        ("wall_push", C.c_double * 6),
        ("wall_mass", C.c_double * 6),
        ("domains", C.c_int64 * 3),
        ("parallel_redraw", C.c_int64),
        ("merge_last_colour", C.c_int64),
    ]


class cd_solve_stats(C.Structure):
    _fields_ = [
        ("sweeps", C.c_int64),
        ("converged", C.c_int64),
        ("residual", C.c_double),
        ("r_avg", C.c_double),
        ("n_contacts", C.c_int64),
        ("n_colours", C.c_int64),
        ("wall_force", C.c_double * 6),
        ("n_phases", C.c_int64),
    ]

    def as_dict(self):
        return {"sweeps": int(self.sweeps), "converged": bool(self.converged), "residual": float(self.residual),
                "r_avg": float(self.r_avg), "n_contacts": int(self.n_contacts), "n_colours": int(self.n_colours),
                "wall_force": [float(v) for v in self.wall_force], "n_phases": int(self.n_phases)}


class cd_step_stats(C.Structure):
    _fields_ = [
        ("steps_done", C.c_int64),
        ("total_sweeps", C.c_int64),
        ("total_contact_updates", C.c_int64),
        ("max_sweeps_in_step", C.c_int64),
        ("n_not_converged", C.c_int64),
        ("kernel_launches", C.c_int64),
        ("phase_ms", C.c_double * 4),
        ("last", cd_solve_stats),
    ]

    def as_dict(self):
        return {"steps_done": int(self.steps_done), "total_sweeps": int(self.total_sweeps),
                "total_contact_updates": int(self.total_contact_updates),
                "max_sweeps_in_step": int(self.max_sweeps_in_step), "n_not_converged": int(self.n_not_converged),
                "kernel_launches": int(self.kernel_launches),
                "phase_ms": {"detect": float(self.phase_ms[0]), "colour_order_pack": float(self.phase_ms[1]),
                             "sweep": float(self.phase_ms[2]), "integrate": float(self.phase_ms[3])},
                "last": self.last.as_dict()}


class cd_packing_stats(C.Structure):
    _fields_ = [
        ("sweeps", C.c_int64),
        ("converged", C.c_int64),
        ("residual", C.c_double),
        ("r_avg", C.c_double),
        ("n_contacts", C.c_int64),
        ("wall_force", C.c_double * 6),
        ("wall_pos", C.c_double * 6),
    ]

    def as_dict(self):
        return {"sweeps": int(self.sweeps), "converged": bool(self.converged), "residual": float(self.residual),
                "r_avg": float(self.r_avg), "n_contacts": int(self.n_contacts),
                "wall_force": [float(v) for v in self.wall_force], "wall_pos": [float(v) for v in self.wall_pos]}


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every entry point declared in include/cd_api.h
_P = C.c_void_p
class cd_adjoint_stats(C.Structure):
    _fields_ = [
        ("sweeps", C.c_int64),
        ("converged", C.c_int64),
        ("residual", C.c_double),
        ("n_contacts", C.c_int64),
        ("n_open", C.c_int64),
        ("n_stick", C.c_int64),
        ("n_slide", C.c_int64),
        ("dL_dmu", C.c_double),
        ("kernel_launches", C.c_int64),
        ("n_rows", C.c_int64),
        ("n_dof", C.c_int64),
        ("diverged", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SIGNATURES = [
    ("cd_create_system", C.c_int, [C.POINTER(cd_params), C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                   C.POINTER(_P)]),
    ("cd_create_batch", C.c_int, [C.POINTER(cd_params), C.c_int64, C.POINTER(C.c_int64), _P, _P, _P, _P, _P, _P, _P,
                                  _P, _P, C.POINTER(_P)]),
    ("cd_workspace_size", C.c_int, [_P, C.POINTER(C.c_size_t)]),
    ("cd_set_workspace", C.c_int, [_P, _P, C.c_size_t]),
    ("cd_detect_contacts", C.c_int, [_P, C.POINTER(C.c_int64)]),
    ("cd_set_contacts", C.c_int, [_P, C.c_int64, _P, _P]),
    ("cd_solve_contacts", C.c_int, [_P, C.POINTER(cd_solve_stats)]),
    ("cd_step", C.c_int, [_P, C.c_int64, C.POINTER(cd_step_stats)]),
    ("cd_get_contacts", C.c_int, [_P, C.POINTER(C.c_int64), _P, _P, _P, _P, _P]),
    ("cd_get_walls", C.c_int, [_P, C.POINTER(C.c_double)]),
    ("cd_get_packing_stats", C.c_int, [_P, C.c_int64, C.c_int64, C.POINTER(cd_packing_stats)]),
    ("cd_force_orientation", C.c_int, [_P, C.c_int64, C.POINTER(C.c_int64)]),
    ("cd_stress_profile", C.c_int, [_P, C.c_int64, C.c_double, C.c_double, C.c_int64, C.POINTER(C.c_double)]),
    ("cd_upload_state", C.c_int, [_P, _P, _P, _P]),
    ("cd_download_state", C.c_int, [_P, _P, _P, _P]),
    ("cd_detect_contacts_noalloc", C.c_int, [C.POINTER(cd_params), C.c_int64, _P, _P, _P, _P, C.c_int64, _P, _P,
                                             _P, C.POINTER(C.c_int64), _P]),
    ("cd_adjoint_step", C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_double), _P, _P, _P, C.c_double, C.c_int64,
                                  C.POINTER(cd_adjoint_stats)]),
    ("cd_checkpoint_size", C.c_int, [_P, C.POINTER(C.c_size_t)]),
    ("cd_save_checkpoint", C.c_int, [_P, _P, C.c_size_t]),
    ("cd_load_checkpoint", C.c_int, [_P, _P, C.c_size_t]),
    ("cd_selfcheck_wait_bound", C.c_int, [_P, C.c_size_t, _P, C.POINTER(C.c_double)]),
    ("cd_destroy_system", None, [_P]),
    ("cd_last_error", C.c_char_p, [_P]),
]


def lib():
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'` on a machine with nvcc")
            L = C.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(sysptr, status, allow=(CD_OK,)):
    if status in allow:
        return status
    msg = lib().cd_last_error(sysptr)
    raise CDError(status, msg.decode() if msg else "")


# --- one-to-one wrappers of the C entry points -------------------------------

def cd_create_system(params: cd_params, n, pos, vel, omega, theta, radius, inv_mass, inv_inertia, f_ext, stream):
    out = _P()
    ptr = lambda t: None if t is None else t.data_ptr()
    st = lib().cd_create_system(C.byref(params), int(n), ptr(pos), ptr(vel), ptr(omega), ptr(theta), ptr(radius),
                                ptr(inv_mass), ptr(inv_inertia), ptr(f_ext), stream, C.byref(out))
    _check(None, st)
    return out


def cd_create_batch(params_list, offsets, pos, vel, omega, theta, radius, inv_mass, inv_inertia, f_ext, stream):
    out = _P()
    ptr = lambda t: None if t is None else t.data_ptr()
    arr = (cd_params * len(params_list))(*params_list)
    offs = (C.c_int64 * len(offsets))(*[int(o) for o in offsets])
    st = lib().cd_create_batch(arr, len(params_list), offs, ptr(pos), ptr(vel), ptr(omega), ptr(theta), ptr(radius),
                               ptr(inv_mass), ptr(inv_inertia), ptr(f_ext), stream, C.byref(out))
    _check(None, st)
    return out


def cd_get_packing_stats(sysptr, first, count):
    arr = (cd_packing_stats * max(count, 1))()
    _check(sysptr, lib().cd_get_packing_stats(sysptr, int(first), int(count), arr))
    return [arr[i].as_dict() for i in range(count)]


def cd_force_orientation(sysptr, nbins=18) -> np.ndarray:
    out = (C.c_int64 * nbins)()
    _check(sysptr, lib().cd_force_orientation(sysptr, int(nbins), out))
    return np.array(list(out), dtype=np.int64)


def cd_stress_profile(sysptr, axis, lo, width, nstripes) -> np.ndarray:
    out = (C.c_double * nstripes)()
    _check(sysptr, lib().cd_stress_profile(sysptr, int(axis), float(lo), float(width), int(nstripes), out))
    return np.array(list(out))


def cd_workspace_size(sysptr) -> int:
    b = C.c_size_t()
    _check(sysptr, lib().cd_workspace_size(sysptr, C.byref(b)))
    return int(b.value)


def cd_set_workspace(sysptr, buf: torch.Tensor):
    _check(sysptr, lib().cd_set_workspace(sysptr, buf.data_ptr(), buf.numel() * buf.element_size()))


def cd_detect_contacts(sysptr) -> int:
    nc = C.c_int64()
    _check(sysptr, lib().cd_detect_contacts(sysptr, C.byref(nc)))
    return int(nc.value)


def cd_set_contacts(sysptr, pairs: torch.Tensor, impulses=None):
    nc = int(pairs.shape[0])
    _check(sysptr, lib().cd_set_contacts(sysptr, nc, pairs.data_ptr() if nc else None,
                                         None if impulses is None else impulses.data_ptr()))


def cd_solve_contacts(sysptr) -> dict:
    st = cd_solve_stats()
    _check(sysptr, lib().cd_solve_contacts(sysptr, C.byref(st)), allow=(CD_OK, CD_ERR_NOT_CONVERGED))
    return st.as_dict()


def cd_step(sysptr, n_steps: int, stats: bool = True):
    st = cd_step_stats()
    _check(sysptr, lib().cd_step(sysptr, int(n_steps), C.byref(st) if stats else None),
           allow=(CD_OK, CD_ERR_NOT_CONVERGED))
    return st.as_dict() if stats else None


def cd_get_contacts(sysptr, pairs, normal, gap, impulse, colour) -> int:
    nc = C.c_int64()
    ptr = lambda t: None if t is None else t.data_ptr()
    _check(sysptr, lib().cd_get_contacts(sysptr, C.byref(nc), ptr(pairs), ptr(normal), ptr(gap), ptr(impulse),
                                         ptr(colour)))
    return int(nc.value)


def cd_get_walls(sysptr) -> np.ndarray:
    out = (C.c_double * 6)()
    _check(sysptr, lib().cd_get_walls(sysptr, out))
    return np.array(list(out))


def cd_upload_state(sysptr, pos_host, vel_host, omega_host):
    ptr = lambda a: None if a is None else (a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data)
    _check(sysptr, lib().cd_upload_state(sysptr, ptr(pos_host), ptr(vel_host), ptr(omega_host)))


def cd_download_state(sysptr, pos_host, vel_host, omega_host):
    ptr = lambda a: None if a is None else (a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data)
    _check(sysptr, lib().cd_download_state(sysptr, ptr(pos_host), ptr(vel_host), ptr(omega_host)))


def cd_detect_contacts_noalloc(params: cd_params, n, pos, radius, inv_mass, inv_inertia, max_contacts, pairs,
                               normal, gap, stream) -> int:
    """Detection without a system or workspace (library-held scratch; see
    cd_api.h).  Checks the tensors first (dtype, contiguity, device, room for
    max_contacts rows: the kernels write through the raw pointers).  On
    CD_ERR_CAPACITY the raised CDError carries the number of contacts needed
    in its `needed` attribute, so a caller can resize and call again."""
    dim = int(params.dim)
    need = [(pos, torch.float64, n * dim, "pos"), (radius, torch.float64, n, "radius"),
            (inv_mass, torch.float64, n, "inv_mass"), (inv_inertia, torch.float64, n, "inv_inertia")]
    if max_contacts > 0 or pairs is not None:
        need += [(pairs, torch.int32, 2 * max_contacts, "pairs"), (normal, torch.float64, 3 * max_contacts, "normal"),
                 (gap, torch.float64, max_contacts, "gap")]
    for t, dt, cnt, name in need:
        if t is None:
            raise ValueError(f"{name} is required")
        if t.dtype != dt or not t.is_contiguous() or t.device != pos.device or t.device.type != "cuda":
            raise ValueError(f"{name} must be a contiguous {dt} tensor on {pos.device}")
        if t.numel() < cnt:
            raise ValueError(f"{name} holds {t.numel()} elements, {cnt} needed")
    nc = C.c_int64()
    ptr = lambda t: None if t is None else t.data_ptr()
    st = lib().cd_detect_contacts_noalloc(C.byref(params), int(n), ptr(pos), ptr(radius), ptr(inv_mass),
                                          ptr(inv_inertia), int(max_contacts), ptr(pairs), ptr(normal), ptr(gap),
                                          C.byref(nc), stream)
    try:
        _check(None, st)
    except CDError as e:
        if e.status == CD_ERR_CAPACITY:
            e.needed = int(nc.value)
        raise
    return int(nc.value)


def cd_adjoint_step(sysptr, dL_dpos, dL_dvel, dL_domega, dL_dwall_force, out_pos, out_vel, out_omega, alpha,
                    max_sweeps) -> dict:
    st = cd_adjoint_stats()
    wf = None
    if dL_dwall_force is not None:
        wf = (C.c_double * 6)(*[float(x) for x in np.asarray(dL_dwall_force, dtype=np.float64).reshape(6)])
    _check(sysptr, lib().cd_adjoint_step(sysptr, dL_dpos.data_ptr(), dL_dvel.data_ptr(), dL_domega.data_ptr(), wf,
                                         out_pos.data_ptr(), out_vel.data_ptr(), out_omega.data_ptr(), float(alpha),
                                         int(max_sweeps), C.byref(st)),
           allow=(CD_OK, CD_ERR_NOT_CONVERGED))
    return st.as_dict()


def cd_checkpoint_size(sysptr) -> int:
    b = C.c_size_t()
    _check(sysptr, lib().cd_checkpoint_size(sysptr, C.byref(b)))
    return int(b.value)


def cd_save_checkpoint(sysptr, buf: torch.Tensor):
    _check(sysptr, lib().cd_save_checkpoint(sysptr, buf.data_ptr(), buf.numel() * buf.element_size()))


def cd_load_checkpoint(sysptr, buf: torch.Tensor):
    _check(sysptr, lib().cd_load_checkpoint(sysptr, buf.data_ptr(), buf.numel() * buf.element_size()))


def cd_selfcheck_wait_bound(buf: torch.Tensor, stream) -> float:
    """Runs the bounded-wait self-check on `stream`; returns the kernel's
    duration in ms (raises CDError if the bound did not fire)."""
    ms = C.c_double()
    _check(None, lib().cd_selfcheck_wait_bound(buf.data_ptr(), buf.numel() * buf.element_size(), stream,
                                               C.byref(ms)))
    return float(ms.value)


def cd_destroy_system(sysptr):
    lib().cd_destroy_system(sysptr)


def cd_last_error(sysptr=None) -> str:
    m = lib().cd_last_error(sysptr)
    return m.decode() if m else ""


# --- convenience object ----------------------------------------------------------

def make_params(wl, precision=CD_FP64, criterion=CD_CONV_GLOBAL_REL, max_contacts=None, warm_start=1, rotations=1,
                seed=None, max_sweeps=None, alpha=None, timing=0,
                parallel_p=0.0, tape_steps=0, adjoint_compliance=0.0, use_graph=0, sweep_threads=0,
                sweep_blocks_per_sm=0, domains=(1, 1, 1), merge_last_colour=4, parallel_redraw=0) -> cd_params:
    p = cd_params()
    p.dim = wl.dim
    p.precision = precision
    p.dt = wl.dt
    p.mu = wl.mu
    for k in range(3):
        p.gravity[k] = wl.gravity[k]
        p.box_lo[k] = wl.box_lo[k]
        p.box_hi[k] = wl.box_hi[k]
        p.periodic[k] = int(wl.periodic[k])
    p.wall_mask = int(wl.wall_mask)
    wp = np.asarray(wl.wall_pos, dtype=np.float64).reshape(6)
    wv = np.asarray(wl.wall_vel, dtype=np.float64).reshape(18)
    for k in range(6):
        p.wall_pos[k] = float(wp[k])
    for k in range(18):
        p.wall_vel[k] = float(wv[k])
    p.delta = wl.delta
    p.alpha = wl.alpha if alpha is None else alpha
    p.criterion = criterion
    p.max_sweeps = wl.max_sweeps if max_sweeps is None else max_sweeps
    p.warm_start = int(warm_start)
    p.rotations = int(rotations)
    p.seed = int(wl.seed if seed is None else seed) & (2**64 - 1)
    p.max_contacts = int(max_contacts if max_contacts is not None else max(64, 6 * wl.n))
    p.timing = int(timing)
    p.parallel_p = float(parallel_p)
    p.tape_steps = int(tape_steps)
    p.adjoint_compliance = float(adjoint_compliance)
    p.use_graph = int(use_graph)
    p.sweep_threads = int(sweep_threads)
    p.sweep_blocks_per_sm = int(sweep_blocks_per_sm)
    push = np.asarray(getattr(wl, "wall_push", np.zeros(6)), dtype=np.float64).reshape(6)
    mass = np.asarray(getattr(wl, "wall_mass", np.zeros(6)), dtype=np.float64).reshape(6)
    for k in range(6):
        p.wall_push[k] = float(push[k])
        p.wall_mass[k] = float(mass[k])
    for k in range(3):
        p.domains[k] = int(domains[k])
    p.merge_last_colour = int(merge_last_colour)
    p.parallel_redraw = int(parallel_redraw)
    return p


def concat_workloads(batch):
    """One Workload holding the particles of all packings (parameters of the
    first); the packings' own parameters go to cd_create_batch separately."""
    import dataclasses
    w0 = batch[0]
    cat = lambda name: np.concatenate([np.asarray(getattr(b, name)) for b in batch], axis=0)
    return dataclasses.replace(w0, x=cat("x"), v=cat("v"), w=cat("w"), r=cat("r"), inv_m=cat("inv_m"),
                               inv_I=cat("inv_I"))


class CDSystem:
    """A CD system over torch-owned device tensors (FP64 state, SoA layouts of cd_api.h)."""

    def __init__(self, wl, device="cuda", f_ext=None, stream=None, batch=None, **param_kw):
        """wl: one Workload, or with batch=[Workload, ...] the list of packings
        (wl is then ignored and the packings are concatenated)."""
        if batch is not None:
            wl = concat_workloads(batch)
            self.packings = batch
            self.n_packings = len(batch)
        self.wl = wl
        self.dim = wl.dim
        self.n = wl.n
        self.device = torch.device(device)
        dd = dict(dtype=torch.float64, device=self.device)
        self.pos = torch.as_tensor(np.ascontiguousarray(wl.x).reshape(-1), **dd).clone()
        self.vel = torch.as_tensor(np.ascontiguousarray(wl.v).reshape(-1), **dd).clone()
        self.omega = torch.as_tensor(np.ascontiguousarray(wl.w).reshape(-1), **dd).clone()
        self.theta = torch.zeros(self.n, **dd) if wl.dim == 2 else None
        self.radius = torch.as_tensor(wl.r, **dd).clone()
        self.inv_mass = torch.as_tensor(wl.inv_m, **dd).clone()
        self.inv_inertia = torch.as_tensor(wl.inv_I, **dd).clone()
        self.f_ext = None if f_ext is None else torch.as_tensor(np.asarray(f_ext).reshape(-1), **dd).clone()
        self.pw = 2 if wl.dim == 2 else 4
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if batch is None:
            self.params = make_params(wl, **param_kw)
            self._h = cd_create_system(self.params, self.n, self.pos, self.vel, self.omega, self.theta, self.radius,
                                       self.inv_mass, self.inv_inertia, self.f_ext, self.stream.cuda_stream)
        else:
            total = sum(b.n for b in batch)
            kw = dict(param_kw)
            kw.setdefault("max_contacts", max(64, 6 * total))
            self.params = [make_params(b, **kw) for b in batch]
            self.offsets = np.concatenate([[0], np.cumsum([b.n for b in batch])]).astype(np.int64)
            self._h = cd_create_batch(self.params, self.offsets, self.pos, self.vel, self.omega, self.theta,
                                      self.radius, self.inv_mass, self.inv_inertia, self.f_ext,
                                      self.stream.cuda_stream)
        nbytes = cd_workspace_size(self._h)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws_view = self.workspace[off: off + nbytes]
        cd_set_workspace(self._h, self._ws_view)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                cd_destroy_system(h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self):
        return self._h

    def detect_contacts(self) -> int:
        return cd_detect_contacts(self._h)

    def set_contacts(self, pairs, impulses=None):
        pairs = torch.as_tensor(np.asarray(pairs, dtype=np.int32).reshape(-1, 2), device=self.device).contiguous()
        imp = None
        if impulses is not None:
            imp = torch.as_tensor(np.asarray(impulses, dtype=np.float64).reshape(-1, self.pw),
                                  device=self.device).contiguous()
        cd_set_contacts(self._h, pairs, imp)

    def solve_contacts(self) -> dict:
        return cd_solve_contacts(self._h)

    def step(self, n_steps=1, stats=True):
        return cd_step(self._h, n_steps, stats)

    def contacts(self) -> dict:
        """Current contact set in key order, as numpy arrays."""
        nc = cd_get_contacts(self._h, None, None, None, None, None)
        m = max(nc, 1)
        pairs = torch.empty((m, 2), dtype=torch.int32, device=self.device)
        normal = torch.empty((m, 3), dtype=torch.float64, device=self.device)
        gap = torch.empty(m, dtype=torch.float64, device=self.device)
        imp = torch.empty((m, self.pw), dtype=torch.float64, device=self.device)
        col = torch.empty(m, dtype=torch.int32, device=self.device)
        nc = cd_get_contacts(self._h, pairs, normal, gap, imp, col)
        return {"pairs": pairs[:nc].cpu().numpy(), "normal": normal[:nc].cpu().numpy(), "gap": gap[:nc].cpu().numpy(),
                "impulse": imp[:nc].cpu().numpy(), "colour": col[:nc].cpu().numpy()}

    def walls(self) -> np.ndarray:
        return cd_get_walls(self._h)

    def force_orientation(self, nbins=18):
        return cd_force_orientation(self._h, nbins)

    def stress_profile(self, axis, lo, width, nstripes):
        return cd_stress_profile(self._h, axis, lo, width, nstripes)

    def adjoint_step(self, dL_dpos, dL_dvel, dL_domega, alpha=1e-13, max_sweeps=100000, dL_dwall_force=None):
        """Gradients with respect to the input state of the most recent
        recorded step, given those of its output state (device tensors of
        the state's shapes) and optionally of its 6 wall forces; returns
        (dL_dpos, dL_dvel, dL_domega, stats)."""
        gx = torch.empty_like(self.pos)
        gv = torch.empty_like(self.vel)
        gw = torch.empty_like(self.omega)
        args = [t.contiguous().to(device=self.device, dtype=torch.float64).reshape(-1)
                for t in (dL_dpos, dL_dvel, dL_domega)]
        st = cd_adjoint_step(self._h, *args, dL_dwall_force, gx, gv, gw, alpha, max_sweeps)
        return gx, gv, gw, st

    def new_checkpoint(self) -> torch.Tensor:
        """A device buffer (256-byte aligned view) for save/load_checkpoint."""
        nbytes = cd_checkpoint_size(self._h)
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-raw.data_ptr()) % 256
        return raw[off: off + nbytes]

    def save_checkpoint(self, buf=None) -> torch.Tensor:
        buf = self.new_checkpoint() if buf is None else buf
        cd_save_checkpoint(self._h, buf)
        return buf

    def load_checkpoint(self, buf):
        cd_load_checkpoint(self._h, buf)

    def packing_stats(self):
        return cd_get_packing_stats(self._h, 0, getattr(self, "n_packings", 1))

    def state(self) -> dict:
        torch.cuda.synchronize(self.device)
        return {"x": self.pos.cpu().numpy().reshape(self.n, self.dim),
                "v": self.vel.cpu().numpy().reshape(self.n, self.dim),
                "w": self.omega.cpu().numpy().reshape(self.n, -1) if self.dim == 3 else self.omega.cpu().numpy(),
                "theta": None if self.theta is None else self.theta.cpu().numpy()}
