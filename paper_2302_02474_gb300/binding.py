"""ctypes binding of the TILD C ABI (include/tild.h).

Argument marshalling only: every step of the method runs in the CUDA
library. Functions keep the C names; ``Tild`` wraps one context for
convenience (numpy arrays are host buffers, CUDA torch tensors device
buffers). There is no CPU fallback: loading fails loudly when the library
has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from ._build import LIB_PATH

TILD_OK = 0
TILD_EINVAL = -1
TILD_ENOMEM = -2
TILD_EUNSUPPORTED = -3
TILD_EDEVICE = -4
TILD_ENAN = -5
TILD_ESTATE = -6
TILD_ETIMEOUT = -7

TILD_FP32, TILD_FP64 = 0, 1
TILD_DTYPE_F32, TILD_DTYPE_F64 = 0, 1
TILD_HOST, TILD_DEVICE = 0, 1
TILD_COMPUTE_ENERGY, TILD_COMPUTE_FORCES = 1, 2
TILD_LAYOUT_AOS, TILD_LAYOUT_SOA = 0, 1

STATUS_NAMES = {0: "TILD_OK", -1: "TILD_EINVAL", -2: "TILD_ENOMEM", -3: "TILD_EUNSUPPORTED", -4: "TILD_EDEVICE",
                -5: "TILD_ENAN", -6: "TILD_ESTATE", -7: "TILD_ETIMEOUT"}


class tild_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double * 3), ("n", ctypes.c_int * 3), ("pmeorder", ctypes.c_int),
                ("precision", ctypes.c_int), ("seed", ctypes.c_uint64), ("sort_every", ctypes.c_int)]


class tild_moltype(ctypes.Structure):
    _fields_ = [("n_chains", ctypes.c_int64), ("N", ctypes.c_int), ("n_a", ctypes.c_int)]


class tild_energy_grad(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("energy", "e_bond", "e_chi", "e_kappa", "dU_dchi", "dU_dkappa", "dU_da",
                                               "e_elec")]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class tild_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class tild_energy(ctypes.Structure):
    _fields_ = [("e_bond", ctypes.c_double), ("e_chi", ctypes.c_double), ("e_kappa", ctypes.c_double),
                ("kinetic", ctypes.c_double), ("net_force", ctypes.c_double * 3), ("e_elec", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_SIGS = {
    "tild_create": [ctypes.POINTER(tild_params), ctypes.POINTER(_P)],
    "tild_create_with_allocator": [ctypes.POINTER(tild_params), ctypes.POINTER(tild_allocator), ctypes.POINTER(_P)],
    "tild_set_species": [_P, _I, _P],
    "tild_set_bonds": [_P, _I64, _P],
    "tild_set_chi_matrix": [_P, _P],
    "tild_set_layout": [_P, _I],
    "tild_destroy": [_P],
    "tild_set_chains": [_P, _I, ctypes.POINTER(tild_moltype), ctypes.c_double],
    "tild_set_interactions": [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double],
    "tild_set_integrator": [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double],
    "tild_set_integrator_scheme": [_P, ctypes.c_int],
    "tild_set_force_method": [_P, ctypes.c_int],
    "tild_set_electrostatics": [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double],
    "tild_force_vjp": [_P, _P, _P, _I, _I, ctypes.POINTER(ctypes.c_double)],
    "tild_density_vjp": [_P, _P, _P, _I, _I],
    "tild_autotune": [_P, _I64, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)],
    "tild_get_launch_shapes": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "tild_set_launch_shapes": [_P, _I, _I],
    "tild_trajectory_vjp": [_P, _I64, _I, _P, _P, _I, _I, _P, _P, ctypes.POINTER(ctypes.c_double)],
    "tild_set_stream": [_P, _P],
    "tild_set_positions": [_P, _P, _I, _I],
    "tild_init_velocities": [_P],
    "tild_set_velocities": [_P, _P, _I, _I],
    "tild_step": [_P, _I64],
    "tild_synchronize": [_P],
    "tild_compute": [_P, ctypes.c_uint, ctypes.POINTER(tild_energy), _P, _I, _I],
    "tild_energy_gradient": [_P, ctypes.POINTER(tild_energy_grad), _P, _I, _I],
    "tild_get_positions": [_P, _P, _I, _I],
    "tild_get_velocities": [_P, _P, _I, _I],
    "tild_get_density": [_P, _P, _I, _I],
    "tild_get_spectrum": [_P, _P, _I, _I],
    "tild_get_field_gradient": [_P, _P, _I, _I],
    "tild_get_step": [_P, ctypes.POINTER(_I64)],
    "tild_state_bytes": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "tild_get_state": [_P, _P, ctypes.c_size_t, _I],
    "tild_set_state": [_P, _P, ctypes.c_size_t, _I],
    "tild_profile_steps": [_P, _I, ctypes.POINTER(ctypes.c_double)],
    "tild_launches_per_steps": [_P, _I64, ctypes.POINTER(_I64)],
    "tild_spread_density_noalloc": [_P, _P, _I64, ctypes.c_double, _I, _I, _P, _P],
    "tild_batch_create": [_I, ctypes.POINTER(_P), ctypes.POINTER(_P)],
    "tild_batch_step": [_P, _I64],
    "tild_batch_synchronize": [_P],
    "tild_batch_launches_per_steps": [_P, _I64, ctypes.POINTER(_I64)],
    "tild_batch_destroy": [_P],
    "tild_batch_is_persistent": [_P, ctypes.POINTER(_I)],
    "tild_batch_set_wait_limit": [_P, _I64, _I],
    "tild_batch_set_persistent": [_P, _I],
    "tild_batch_autotune": [_P, _I64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I)],
}

_lib: Optional[ctypes.CDLL] = None


def library_path() -> str:
    return os.environ.get("TILD_LIBRARY", LIB_PATH)


def load() -> ctypes.CDLL:
    """Load libtild.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"TILD CUDA library not found at {path}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.tild_last_error.argtypes = [_P]
    lib.tild_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


class TildError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, ctx=None) -> None:
    if status != TILD_OK:
        msg = load().tild_last_error(ctx).decode()
        raise TildError(status, msg)


def declared_symbols() -> Sequence[str]:
    return list(_SIGS) + ["tild_last_error"]


# ------------------------------------------------------------------ helpers


def _buffer(arr, n_elems: int):
    """(pointer, dtype code, where code, keepalive) for a numpy array or torch tensor."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(arr, torch.Tensor):
        if not arr.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if arr.dtype not in (torch.float32, torch.float64):
            raise ValueError("tensor dtype must be float32 or float64")
        if arr.numel() != n_elems:
            raise ValueError(f"expected {n_elems} elements, got {arr.numel()}")
        code = TILD_DTYPE_F32 if arr.dtype == torch.float32 else TILD_DTYPE_F64
        where = TILD_DEVICE if arr.is_cuda else TILD_HOST
        return ctypes.c_void_p(arr.data_ptr()), code, where, arr
    a = np.ascontiguousarray(arr)
    if a.dtype not in (np.float32, np.float64):
        a = a.astype(np.float64)
    if a.size != n_elems:
        raise ValueError(f"expected {n_elems} elements, got {a.size}")
    code = TILD_DTYPE_F32 if a.dtype == np.float32 else TILD_DTYPE_F64
    return ctypes.c_void_p(a.ctypes.data), code, TILD_HOST, a


class TorchAllocator:
    """Device memory of a context from PyTorch's caching allocator, for
    tild_create_with_allocator. Counts live blocks and bytes (for tests)."""

    def __init__(self, device: int = 0):
        import torch

        self.torch = torch
        self.device = device
        self.live = {}
        self.n_alloc = 0
        self.fail_after = None  # tests: refuse the allocation after this many

        def _alloc(nbytes, _user):
            if self.fail_after is not None and self.n_alloc >= self.fail_after:
                return None
            ptr = self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device)
            self.live[ptr] = int(nbytes)
            self.n_alloc += 1
            return ptr

        def _free(ptr, _nbytes, _user):
            self.live.pop(ptr, None)
            self.torch.cuda.caching_allocator_delete(ptr)

        self._fns = (ALLOC_FN(_alloc), FREE_FN(_free))  # keep the callbacks alive
        self.struct = tild_allocator(self._fns[0], self._fns[1], None)

    @property
    def live_bytes(self) -> int:
        return sum(self.live.values())


class Tild:
    """One TILD context (thin wrapper over the C ABI)."""

    def __init__(self, L: float, n: int, pmeorder: int = 1, precision: str = "fp32", seed: int = 0,
                 sort_every: int = 0, allocator: Optional[TorchAllocator] = None, dim: int = 3):
        """A context for a cubic box (dim=3) or a square box with an n x n
        grid (dim=2; per-bead arrays keep three components, z unused)."""
        lib = load()
        p = tild_params()
        p.L[:] = [L, L, L]
        p.n[:] = [n, n, n] if dim == 3 else [n, n, 1]
        self.dim = dim
        self.nz = n if dim == 3 else 1
        p.pmeorder = pmeorder
        p.precision = TILD_FP32 if precision == "fp32" else TILD_FP64
        p.seed = seed
        p.sort_every = sort_every
        ctx = ctypes.c_void_p()
        self.allocator = allocator  # must outlive the context
        if allocator is not None:
            check(lib.tild_create_with_allocator(ctypes.byref(p), ctypes.byref(allocator.struct), ctypes.byref(ctx)),
                  None)
        else:
            check(lib.tild_create(ctypes.byref(p), ctypes.byref(ctx)), None)
        self.ctx = ctx
        self.lib = lib
        self.n = n
        self.L = L
        self.np_dtype = np.float32 if precision == "fp32" else np.float64
        self.n_beads = 0
        self.n_species = 2
        self.layout = "aos"
        self.integrator = (0.005, 1.0, 1.0, 1.0)  # dt, friction, kT, mass (the library defaults)
        self.scheme = "gjf"
        self.force_method = "ik"
        self.interactions = None  # (chi, kappa, a) once set

    @classmethod
    def from_spec(cls, spec, sort_every: int = 0, precision: Optional[str] = None) -> "Tild":
        t = cls(spec.L, spec.n, spec.pmeorder, precision or spec.precision, spec.dyn_seed, sort_every)
        t.set_chains([(m.n_chains, m.N, m.n_a) for m in spec.moltypes], spec.b)
        t.set_interactions(spec.chi, spec.kappa, spec.a)
        t.set_integrator(spec.dt, spec.friction, spec.kT, spec.mass)
        return t

    def close(self) -> None:
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.tild_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _chk(self, st: int) -> None:
        check(st, self.ctx)

    def set_chains(self, types, b: float = 1.0) -> None:
        arr = (tild_moltype * len(types))()
        total = 0
        for i, (nc, N, na) in enumerate(types):
            arr[i].n_chains, arr[i].N, arr[i].n_a = nc, N, na
            total += nc * N
        self._chk(self.lib.tild_set_chains(self.ctx, len(types), arr, b))
        self.n_beads = total
        self.n_species = 2

    def set_species(self, n_species: int, species=None) -> None:
        """Species count (1..4) and, optionally, every bead's species (int
        array by bead id); None keeps the chains' A/B pattern."""
        ptr = ctypes.c_void_p()
        keep = None
        if species is not None:
            keep = np.ascontiguousarray(species, dtype=np.int32)
            if keep.size != self.n_beads:
                raise ValueError("one species per bead")
            ptr = ctypes.c_void_p(keep.ctypes.data)
        self._chk(self.lib.tild_set_species(self.ctx, int(n_species), ptr))
        self.n_species = int(n_species)

    def set_bonds(self, pairs) -> None:
        """Explicit bond list, an (n_bonds, 2) int array of bead ids."""
        a = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        ptr = ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p()
        self._chk(self.lib.tild_set_bonds(self.ctx, int(a.shape[0]), ptr))

    def set_chi_matrix(self, chi) -> None:
        a = np.ascontiguousarray(chi, dtype=np.float64)
        if a.shape != (self.n_species, self.n_species):
            raise ValueError("chi must be n_species x n_species")
        self._chk(self.lib.tild_set_chi_matrix(self.ctx, ctypes.c_void_p(a.ctypes.data)))

    LAYOUTS = {"aos": TILD_LAYOUT_AOS, "soa": TILD_LAYOUT_SOA}

    def set_layout(self, layout: str) -> None:
        """Per-bead vectors as "aos" [n][3] (default) or "soa" [3][n]."""
        self._chk(self.lib.tild_set_layout(self.ctx, self.LAYOUTS[layout]))
        self.layout = layout

    def _vec(self, r):
        if not isinstance(r, np.ndarray):
            return r
        return r.reshape(-1, 3) if self.layout == "aos" else r.reshape(3, -1)

    @property
    def n_pairs(self) -> int:
        return 2 if self.n_species > 2 else 1

    def set_interactions(self, chi: float, kappa: float, a: float) -> None:
        self._chk(self.lib.tild_set_interactions(self.ctx, chi, kappa, a))
        self.interactions = (float(chi), float(kappa), float(a))

    def set_integrator(self, dt: float, friction: float, kT: float, mass: float = 1.0) -> None:
        self._chk(self.lib.tild_set_integrator(self.ctx, dt, friction, kT, mass))
        self.integrator = (float(dt), float(friction), float(kT), float(mass))

    def set_electrostatics(self, q_a: float, q_b: float, bjerrum: float, smear: float) -> None:
        """Per-species charges, Bjerrum length (0: off) and charge spreading
        length of the smeared-charge Coulomb interaction."""
        self._chk(self.lib.tild_set_electrostatics(self.ctx, q_a, q_b, bjerrum, smear))

    FORCE_METHODS = {"ik": 0, "analytic": 1}

    def set_force_method(self, method: str) -> None:
        """Particle-mesh force: "ik" (spectral gradient, default) or
        "analytic" (gradient of the assignment weights on the potentials)."""
        self._chk(self.lib.tild_set_force_method(self.ctx, self.FORCE_METHODS[method]))
        self.force_method = method

    SCHEMES = {"gjf": 0, "em": 1, "vv": 2}

    def set_scheme(self, scheme: str) -> None:
        """Integrator of Sec. "Integrator Class": "gjf" (default), "em"
        (Euler-Maruyama, overdamped) or "vv" (velocity-Verlet + Langevin force)."""
        self._chk(self.lib.tild_set_integrator_scheme(self.ctx, self.SCHEMES[scheme]))
        self.scheme = scheme

    def set_stream(self, stream) -> None:
        handle = getattr(stream, "cuda_stream", stream)
        self._chk(self.lib.tild_set_stream(self.ctx, ctypes.c_void_p(handle or 0)))

    def set_positions(self, xyz) -> None:
        ptr, code, where, _keep = _buffer(xyz, 3 * self.n_beads)
        self._chk(self.lib.tild_set_positions(self.ctx, ptr, code, where))

    def init_velocities(self) -> None:
        self._chk(self.lib.tild_init_velocities(self.ctx))

    def set_velocities(self, v) -> None:
        ptr, code, where, _keep = _buffer(v, 3 * self.n_beads)
        self._chk(self.lib.tild_set_velocities(self.ctx, ptr, code, where))

    def step(self, n: int = 1) -> None:
        self._chk(self.lib.tild_step(self.ctx, int(n)))

    def synchronize(self) -> None:
        self._chk(self.lib.tild_synchronize(self.ctx))

    def _out(self, fn, count: int, out=None, dtype=np.float64):
        if out is None:
            out = np.empty(count, dtype=dtype)
        ptr, code, where, _keep = _buffer(out, count)
        self._chk(fn(self.ctx, ptr, code, where))
        return out

    def positions(self, out=None, dtype=np.float64):
        return self._vec(self._out(self.lib.tild_get_positions, 3 * self.n_beads, out, dtype))

    def velocities(self, out=None, dtype=np.float64):
        return self._vec(self._out(self.lib.tild_get_velocities, 3 * self.n_beads, out, dtype))

    def density(self, out=None, dtype=np.float64):
        S = self.n_species
        r = self._out(self.lib.tild_get_density, S * self.nz * self.n ** 2, out, dtype)
        return r.reshape(S, self.nz, self.n, self.n) if isinstance(r, np.ndarray) else r

    def spectrum(self, out=None, dtype=np.float64):
        """DFT of rho_0 + i rho_1 [kz][ky][kx] (with more than two species,
        [pair][kz][ky][kx])."""
        npr = self.n_pairs
        r = self._out(self.lib.tild_get_spectrum, 2 * npr * self.nz * self.n ** 2, out, dtype)
        if isinstance(r, np.ndarray):
            r = r.reshape(npr, self.nz, self.n, self.n, 2)
            r = r[..., 0] + 1j * r[..., 1]
            return r[0] if npr == 1 else r
        return r

    def field_gradient(self, out=None, dtype=np.float64):
        npr = self.n_pairs
        D = self.dim
        r = self._out(self.lib.tild_get_field_gradient, 2 * D * npr * self.nz * self.n ** 2, out, dtype)
        if isinstance(r, np.ndarray):
            r = r.reshape(npr, D, self.nz, self.n, self.n, 2)
            return r[0] if npr == 1 else r
        return r

    def compute(self, forces: bool = True, energy: bool = True, out=None, dtype=np.float64):
        e = tild_energy()
        what = (TILD_COMPUTE_ENERGY if energy else 0) | (TILD_COMPUTE_FORCES if forces else 0)
        f = None
        ptr, code, where = ctypes.c_void_p(), TILD_DTYPE_F64, TILD_HOST
        if forces:
            f = np.empty(3 * self.n_beads, dtype=dtype) if out is None else out
            ptr, code, where, _keep = _buffer(f, 3 * self.n_beads)
        self._chk(self.lib.tild_compute(self.ctx, what, ctypes.byref(e), ptr, code, where))
        en = {"bond": e.e_bond, "chi": e.e_chi, "kappa": e.e_kappa, "elec": e.e_elec, "kinetic": e.kinetic,
              "net_force": np.array(e.net_force[:])}
        if f is not None:
            f = self._vec(f)
        return f, en

    def force_vjp(self, lam, out=None):
        """(J^T lam by bead id, {"chi", "kappa", "a"}: d(lam . F)/dtheta) for
        the ik force at the current positions; lam is a host array or a
        CUDA tensor of n_beads x 3."""
        n3 = 3 * self.n_beads
        lptr, lcode, lwhere, _k1 = _buffer(lam, n3)
        if out is None:
            out = np.empty(n3, dtype=np.float64 if lcode == TILD_DTYPE_F64 else np.float32)
        optr, ocode, owhere, _k2 = _buffer(out, n3)
        if (ocode, owhere) != (lcode, lwhere):
            raise ValueError("force_vjp: lam and out must share dtype and memory space")
        th = (ctypes.c_double * 3)()
        self._chk(self.lib.tild_force_vjp(self.ctx, lptr, optr, lcode, lwhere, th))
        return self._vec(out), {"chi": th[0], "kappa": th[1], "a": th[2]}

    def density_vjp(self, dL_drho, out=None):
        """d/dr of sum_{K,g} dL_drho[K, z, y, x] rho_K(g) by bead id, for a
        grid adjoint of shape (n_species, n, n, n) (host array or CUDA tensor;
        out is of the same kind and dtype)."""
        cnt = self.n_species * self.nz * self.n ** 2
        pptr, pcode, pwhere, _k1 = _buffer(dL_drho, cnt)
        if out is None:
            out = np.empty(3 * self.n_beads, dtype=np.float64 if pcode == TILD_DTYPE_F64 else np.float32)
        optr, ocode, owhere, _k2 = _buffer(out, 3 * self.n_beads)
        if (ocode, owhere) != (pcode, pwhere):
            raise ValueError("density_vjp: dL_drho and out must share dtype and memory space")
        self._chk(self.lib.tild_density_vjp(self.ctx, pptr, optr, pcode, pwhere))
        return self._vec(out)

    def energy_gradient(self, with_positions: bool = True, out=None, dtype=np.float64):
        """(dict of U, its terms and dU/dchi, dU/dkappa, dU/da; dU/dr or None)."""
        g = tild_energy_grad()
        ptr, code, where, buf = ctypes.c_void_p(), TILD_DTYPE_F64, TILD_HOST, None
        if with_positions:
            buf = np.empty(3 * self.n_beads, dtype=dtype) if out is None else out
            ptr, code, where, _keep = _buffer(buf, 3 * self.n_beads)
        self._chk(self.lib.tild_energy_gradient(self.ctx, ctypes.byref(g), ptr, code, where))
        d = {k: getattr(g, k) for k, _ in tild_energy_grad._fields_}
        return d, (self._vec(buf) if buf is not None else None)

    def step_count(self) -> int:
        s = ctypes.c_int64()
        self._chk(self.lib.tild_get_step(self.ctx, ctypes.byref(s)))
        return s.value

    def state_bytes(self) -> int:
        nb = ctypes.c_size_t()
        self._chk(self.lib.tild_state_bytes(self.ctx, ctypes.byref(nb)))
        return nb.value

    def get_state(self, out=None):
        """Checkpoint blob: bytes (host), or written into `out`, a CUDA uint8
        tensor of state_bytes() elements (device)."""
        nb = self.state_bytes()
        if out is not None:
            if not out.is_cuda or out.numel() < nb or out.element_size() != 1:
                raise ValueError("out must be a CUDA uint8 tensor of state_bytes() elements")
            self._chk(self.lib.tild_get_state(self.ctx, ctypes.c_void_p(out.data_ptr()), nb, TILD_DEVICE))
            return out
        buf = ctypes.create_string_buffer(nb)
        self._chk(self.lib.tild_get_state(self.ctx, buf, nb, TILD_HOST))
        return buf.raw

    def set_state(self, blob) -> None:
        """Restore a blob from get_state (bytes, or a CUDA uint8 tensor)."""
        if isinstance(blob, (bytes, bytearray)):
            buf = ctypes.create_string_buffer(bytes(blob), len(blob))
            self._chk(self.lib.tild_set_state(self.ctx, buf, len(blob), TILD_HOST))
        else:
            self._chk(self.lib.tild_set_state(self.ctx, ctypes.c_void_p(blob.data_ptr()), blob.numel(), TILD_DEVICE))

    AUTOTUNE_PERIODS = (5, 10, 20, 40)

    def autotune(self, trial_steps: int = 160):
        """Pick the fastest re-binning period (results do not depend on it);
        returns (period, {period: ms per step})."""
        k = ctypes.c_int()
        ms = (ctypes.c_double * 4)()
        self._chk(self.lib.tild_autotune(self.ctx, int(trial_steps), ctypes.byref(k), ms))
        return k.value, dict(zip(self.AUTOTUNE_PERIODS, list(ms)))

    def launch_shapes(self):
        """(plane threads, z column tile) of the step's FFT passes."""
        a, b = ctypes.c_int(), ctypes.c_int()
        self._chk(self.lib.tild_get_launch_shapes(self.ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_launch_shapes(self, plane_threads: int, z_columns: int) -> None:
        self._chk(self.lib.tild_set_launch_shapes(self.ctx, int(plane_threads), int(z_columns)))

    def profile_steps(self, n: int):
        ms = (ctypes.c_double * 5)()
        self._chk(self.lib.tild_profile_steps(self.ctx, int(n), ms))
        return list(ms)

    def launches(self, n_steps: int) -> int:
        v = ctypes.c_int64()
        self._chk(self.lib.tild_launches_per_steps(self.ctx, int(n_steps), ctypes.byref(v)))
        return v.value


class TildBatch:
    """Several Tild contexts stepped together (tild_batch_*)."""

    def __init__(self, replicas: Sequence[Tild]):
        lib = load()
        self.replicas = list(replicas)
        arr = (ctypes.c_void_p * len(self.replicas))(*[r.ctx.value for r in self.replicas])
        h = ctypes.c_void_p()
        check(lib.tild_batch_create(len(self.replicas), arr, ctypes.byref(h)), None)
        self.h = h
        self.lib = lib

    def step(self, n: int = 1) -> None:
        check(self.lib.tild_batch_step(self.h, int(n)), None)

    def synchronize(self) -> None:
        check(self.lib.tild_batch_synchronize(self.h), None)

    def launches(self, n_steps: int) -> int:
        v = ctypes.c_int64()
        check(self.lib.tild_batch_launches_per_steps(self.h, int(n_steps), ctypes.byref(v)), None)
        return v.value

    @property
    def persistent(self) -> bool:
        v = ctypes.c_int()
        check(self.lib.tild_batch_is_persistent(self.h, ctypes.byref(v)), None)
        return bool(v.value)

    def set_persistent(self, on: bool) -> None:
        check(self.lib.tild_batch_set_persistent(self.h, 1 if on else 0), None)

    AUTOTUNE_CANDIDATES = ("persistent 2/SM", "persistent 3/SM", "persistent 4/SM", "groups 512", "groups 512 alt-z",
                           "groups 256", "groups 256 alt-z", "groups 128", "groups 128 alt-z")

    def autotune(self, trial_steps: int = 40):
        """Keep the fastest of the persistent kernel and the group launch
        shapes; returns (chosen candidate, {candidate: ms per step})."""
        ms = (ctypes.c_double * 9)()
        ch = ctypes.c_int()
        check(self.lib.tild_batch_autotune(self.h, int(trial_steps), ms, ctypes.byref(ch)), None)
        return self.AUTOTUNE_CANDIDATES[ch.value], dict(zip(self.AUTOTUNE_CANDIDATES, list(ms)))

    def set_wait_limit(self, wait_ns: int, extra: int = 0) -> None:
        """Limit of one barrier wait of the persistent kernel; extra > 0 makes
        every wait unreachable (tests of the time limit)."""
        check(self.lib.tild_batch_set_wait_limit(self.h, int(wait_ns), int(extra)), None)

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.tild_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
