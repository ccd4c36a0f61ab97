"""Python binding of the C ABI in include/gsis.h (argument marshalling only).

Every numerical step runs in libgsis.so.  PyTorch supplies device memory (its
caching allocator, through the allocator callbacks) and the CUDA stream.  If
the shared library is missing the import fails loudly: there is no CPU path.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgsis.so")

GSIS_OK, GSIS_ERR_ARG, GSIS_ERR_STATE, GSIS_ERR_OOM, GSIS_ERR_CUDA = 0, 1, 2, 3, 4
GSIS_ERR_NONFINITE, GSIS_ERR_TIMEOUT, GSIS_ERR_UNSUPPORTED, GSIS_ERR_INTERNAL = 5, 6, 7, 8
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_STATE", "ERR_OOM", "ERR_CUDA", "ERR_NONFINITE", "ERR_TIMEOUT",
                "ERR_UNSUPPORTED", "ERR_INTERNAL"]
DTYPES = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
DTYPE_BYTES = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}
FIELDS = ["rho", "ux", "uy", "uz", "T", "hot_sxx", "hot_syy", "hot_szz", "hot_sxy", "hot_sxz", "hot_syz",
          "hot_qx", "hot_qy", "hot_qz", "kn_gll", "dvm", "wall_q",
          "sxx", "syy", "szz", "sxy", "sxz", "syz", "qx", "qy", "qz", "p",
          "wall_p", "wall_tx", "wall_ty", "wall_tz"]
PHASES = ["adapt", "cell_eq", "sweep", "moments", "macro", "correct", "residual", "presolve"]

EXPORTED = ["gsis_init", "gsis_set_mesh", "gsis_set_velocity_grid", "gsis_iterate", "gsis_moments",
            "gsis_get_vdf", "gsis_debug_set_region", "gsis_last_error", "gsis_free", "gsis_version",
            "gsis_corrected_maxwellian_noalloc", "gsis_iterate_batch", "gsis_batch_info", "gsis_tuning_info",
            "gsis_debug_set_sweep_tile", "gsis_debug_vdf_moments", "gsis_debug_set_macro_path",
            "gsis_probe_fma_peak", "gsis_debug_set_batch_tile", "gsis_two_vdf_reference",
            "gsis_two_vdf_moments", "gsis_sweep_levels"]
MACRO_PATHS = {"auto": 0, "fused": 1, "multi": 2, "persistent": 3, "persistent_stall": 4}


class GsisError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("Kn", ctypes.c_double), ("omega", ctypes.c_double), ("adaptive", ctypes.c_int),
                ("Kn_ref", ctypes.c_double), ("adapt_every", ctypes.c_int), ("wall_layers", ctypes.c_int),
                ("vdf_dtype", ctypes.c_int), ("macro_steps", ctypes.c_int), ("cfl", ctypes.c_double),
                ("k_sub", ctypes.c_int), ("dt", ctypes.c_double), ("tol", ctypes.c_double),
                ("presolve_max_blocks", ctypes.c_int), ("spin_limit", ctypes.c_ulonglong),
                ("relax", ctypes.c_double), ("d_r", ctypes.c_int), ("Z_r", ctypes.c_double),
                ("A", ctypes.c_double * 4)]


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)),
                ("free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)),
                ("user", ctypes.c_void_p)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("ni", ctypes.c_int), ("nj", ctypes.c_int), ("nk", ctypes.c_int), ("dim", ctypes.c_int),
                ("centers", ctypes.POINTER(ctypes.c_double)), ("volumes", ctypes.POINTER(ctypes.c_double)),
                ("S", ctypes.POINTER(ctypes.c_double) * 3), ("xf", ctypes.POINTER(ctypes.c_double) * 3),
                ("bc_type", ctypes.c_int * 6), ("bc_state", (ctypes.c_double * 5) * 6),
                ("W0", ctypes.POINTER(ctypes.c_double))]


class VGridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("reduced", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("total_iterations", ctypes.c_int), ("eps", ctypes.c_double),
                ("converged", ctypes.c_int), ("n_dvm", ctypes.c_longlong), ("n_v", ctypes.c_longlong),
                ("vdf_bytes", ctypes.c_longlong), ("presolve_blocks", ctypes.c_int),
                ("phase_ms", ctypes.c_double * 8), ("sweep_launches", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong)]


_lib = None


def load():
    """Load libgsis.so and declare the ABI (raises if the library is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgsis.so is not built (run __graft_entry__.build() or "
                          "python paper_2501_02245_gb300/build.py); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, c_int, c_double = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.gsis_init.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Allocator), vp, ctypes.POINTER(vp)]
    lib.gsis_set_mesh.argtypes = [vp, ctypes.POINTER(MeshDesc)]
    lib.gsis_set_velocity_grid.argtypes = [vp, ctypes.POINTER(VGridDesc)]
    lib.gsis_iterate.argtypes = [vp, c_int, ctypes.POINTER(Report)]
    lib.gsis_moments.argtypes = [vp, ctypes.c_uint, ctypes.POINTER(c_double), c_int]
    lib.gsis_get_vdf.argtypes = [vp, ctypes.POINTER(c_double), ctypes.POINTER(c_int), ctypes.c_longlong]
    lib.gsis_debug_set_region.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8)]
    lib.gsis_last_error.argtypes = [vp]
    lib.gsis_last_error.restype = ctypes.c_char_p
    lib.gsis_free.argtypes = [vp]
    lib.gsis_free.restype = None
    lib.gsis_version.restype = ctypes.c_char_p
    lib.gsis_corrected_maxwellian_noalloc.argtypes = [vp, c_int, ctypes.POINTER(VGridDesc), vp, vp]
    lib.gsis_corrected_maxwellian_noalloc.restype = c_int
    lib.gsis_iterate_batch.argtypes = [ctypes.POINTER(vp), c_int, c_int, ctypes.POINTER(Report)]
    lib.gsis_batch_info.argtypes = [ctypes.POINTER(vp), c_int]
    lib.gsis_batch_info.restype = ctypes.c_char_p
    lib.gsis_debug_set_sweep_tile.argtypes = [vp, ctypes.c_char_p]
    lib.gsis_debug_set_sweep_tile.restype = c_int
    lib.gsis_debug_vdf_moments.argtypes = [vp, c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_longlong]
    lib.gsis_debug_vdf_moments.restype = c_int
    lib.gsis_debug_set_macro_path.argtypes = [vp, c_int]
    lib.gsis_debug_set_macro_path.restype = c_int
    lib.gsis_debug_set_batch_tile.argtypes = [ctypes.c_char_p]
    lib.gsis_debug_set_batch_tile.restype = c_int
    lib.gsis_probe_fma_peak.argtypes = [c_int, vp, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]
    lib.gsis_probe_fma_peak.restype = c_int
    lib.gsis_two_vdf_reference.argtypes = [vp, vp, c_int, c_int, c_double, ctypes.POINTER(c_double), vp]
    lib.gsis_two_vdf_reference.restype = c_int
    lib.gsis_two_vdf_moments.argtypes = [vp, vp, c_int, c_int, vp]
    lib.gsis_two_vdf_moments.restype = c_int
    ip = ctypes.POINTER(c_int)
    lib.gsis_sweep_levels.argtypes = [c_int, ip, ip, ctypes.POINTER(c_double), ip, ip]
    lib.gsis_sweep_levels.restype = c_int
    lib.gsis_tuning_info.argtypes = [vp]
    lib.gsis_tuning_info.restype = ctypes.c_char_p
    for name in ("gsis_init", "gsis_set_mesh", "gsis_set_velocity_grid", "gsis_iterate", "gsis_moments",
                 "gsis_get_vdf", "gsis_debug_set_region", "gsis_iterate_batch"):
        getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class _TorchAllocator:
    """Allocator callbacks backed by torch's CUDA caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}

        def _alloc(nbytes, stream, user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
            except Exception:
                return None
            self.live[p] = nbytes
            return p

        def _free(ptr, stream, user):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.c_alloc = Allocator._fields_[0][1](_alloc)
        self.c_free = Allocator._fields_[1][1](_free)
        self.struct = Allocator(self.c_alloc, self.c_free, None)


class Solver:
    """One GSIS solve on one GPU.

    params: dict with Kn, omega, adaptive, Kn_ref, adapt_every, wall_layers,
    macro_steps, cfl, k_sub, dt, tol, presolve_max_blocks; vdf_dtype is one of
    f64 / f32 / bf16 / f16.  mesh: object with ni, nj, nk, dim, centers,
    volumes, S[3], xf[3], bc_type, bc_state (numpy, layout of gsis_mesh_desc);
    W0 [ncell, 5]; vgrid: object with n, lo, hi.
    """

    def __init__(self, params, mesh, W0, vgrid, vdf_dtype="f64", stream=None, use_torch_allocator=True,
                 forced_flags=None):
        lib = load()
        self.lib = lib
        self.ctx = ctypes.c_void_p()
        self.vdf_dtype = vdf_dtype
        p = Params(float(params["Kn"]), float(params["omega"]), int(params.get("adaptive", 0)),
                   float(params.get("Kn_ref", 0.0)), int(params.get("adapt_every", 5)),
                   int(params.get("wall_layers", 2)), DTYPES[vdf_dtype], int(params.get("macro_steps", 200)),
                   float(params.get("cfl", 5.0)), int(params.get("k_sub", 2)), float(params.get("dt", 0.0)),
                   float(params.get("tol", 1e-6)), int(params.get("presolve_max_blocks", 0)),
                   int(params.get("spin_limit", 0)),
                   float(params.get("relax", 1.0)), int(params.get("d_r", 0)), float(params.get("Z_r", 0.0)),
                   (ctypes.c_double * 4)(*params.get("A", (0.0, 0.0, 0.0, 0.0))))
        self._alloc = None
        alloc_ptr = None
        stream_ptr = None
        try:
            import torch
            if torch.cuda.is_available():
                dev = torch.cuda.current_device()
                if stream is None:
                    stream = torch.cuda.current_stream(dev)
                stream_ptr = ctypes.c_void_p(stream.cuda_stream)
                if use_torch_allocator:
                    self._alloc = _TorchAllocator(dev)
                    alloc_ptr = ctypes.byref(self._alloc.struct)
        except ImportError:
            pass
        self.stream = stream
        self._check(lib.gsis_init(ctypes.byref(p), alloc_ptr, stream_ptr, ctypes.byref(self.ctx)), init=True)
        self.ncell = mesh.ni * mesh.nj * mesh.nk
        self._set_mesh(mesh, W0)
        self._set_vgrid(vgrid)
        self.nv = 2 * int(vgrid.n[0]) * int(vgrid.n[1]) if getattr(vgrid, "reduced", False) else int(np.prod(vgrid.n))
        if forced_flags is not None:
            fl = np.ascontiguousarray(np.asarray(forced_flags, dtype=np.uint8).reshape(-1))
            self._check(lib.gsis_debug_set_region(self.ctx, fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))

    @classmethod
    def from_case(cls, case, vdf_dtype="f64", stream=None, forced_flags=None, **overrides):
        params = dict(Kn=case.Kn, omega=case.omega, adaptive=int(case.adaptive), Kn_ref=case.Kn_ref,
                      adapt_every=case.adapt_every, wall_layers=case.wall_layers, macro_steps=case.macro_steps,
                      cfl=case.cfl, k_sub=case.k_sub, dt=case.dt, tol=case.tol,
                      presolve_max_blocks=case.presolve_max_blocks, relax=case.relax)
        params.update(overrides)
        return cls(params, case.mesh, case.W0, case.vgrid, vdf_dtype=vdf_dtype, stream=stream,
                   forced_flags=forced_flags)

    # ------------------------------------------------------------------ internals
    def _check(self, status, init=False):
        if status != GSIS_OK:
            msg = "" if init else self.lib.gsis_last_error(self.ctx).decode()
            raise GsisError(status, msg)

    def _set_mesh(self, mesh, W0):
        keep = []

        def arr(a):
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            keep.append(a)
            return a

        md = MeshDesc()
        md.ni, md.nj, md.nk, md.dim = int(mesh.ni), int(mesh.nj), int(mesh.nk), int(mesh.dim)
        md.centers = _dptr(arr(mesh.centers))
        md.volumes = _dptr(arr(mesh.volumes))
        for d in range(3):
            md.S[d] = _dptr(arr(mesh.S[d]))
            md.xf[d] = _dptr(arr(mesh.xf[d]))
        for s in range(6):
            md.bc_type[s] = int(mesh.bc_type[s])
            for q in range(5):
                md.bc_state[s][q] = float(mesh.bc_state[s][q])
        md.W0 = _dptr(arr(W0))
        self._check(self.lib.gsis_set_mesh(self.ctx, ctypes.byref(md)))

    def _set_vgrid(self, vg):
        d = VGridDesc()
        for a in range(3):
            d.n[a], d.lo[a], d.hi[a] = int(vg.n[a]), float(vg.lo[a]), float(vg.hi[a])
        d.reduced = 1 if getattr(vg, "reduced", False) else 0
        self._check(self.lib.gsis_set_velocity_grid(self.ctx, ctypes.byref(d)))

    # ------------------------------------------------------------------ API
    def iterate(self, n):
        rep = Report()
        self._check(self.lib.gsis_iterate(self.ctx, int(n), ctypes.byref(rep)))
        out = {f: getattr(rep, f) for f, _ in Report._fields_ if f != "phase_ms"}
        out["phase_ms"] = {PHASES[i]: rep.phase_ms[i] for i in range(8)}
        return out

    def moments(self, fields=("rho", "ux", "uy", "uz", "T")):
        mask = 0
        for f in fields:
            mask |= 1 << FIELDS.index(f)
        order = [f for f in FIELDS if f in fields]
        out = np.zeros((self.ncell, len(order)))
        self._check(self.lib.gsis_moments(self.ctx, mask, _dptr(out), 0))
        return {f: out[:, i].copy() for i, f in enumerate(order)}

    def W(self):
        m = self.moments()
        return np.stack([m["rho"], m["ux"], m["uy"], m["uz"], m["T"]], axis=1)

    def set_sweep_tile(self, name):
        """Force the kinetic sweep's tile shape (test hook)."""
        self._check(self.lib.gsis_debug_set_sweep_tile(self.ctx, name.encode()))

    def vdf_moments(self, n_dvm, direct):
        """Per-DVM-cell velocity moments of the VDF, [n_dvm, 19] (test hook):
        the ones the last iteration carried forward (direct=False) or a fresh
        reduction over the current VDF (direct=True)."""
        out = np.zeros((n_dvm, 19))
        self._check(self.lib.gsis_debug_vdf_moments(self.ctx, int(bool(direct)), _dptr(out), out.size))
        return out

    def set_macro_path(self, name):
        """Choose the synthetic-solve implementation (test hook): auto, fused,
        multi, persistent, or persistent_stall (a barrier that can only end by
        running out of spin_limit polls)."""
        self._check(self.lib.gsis_debug_set_macro_path(self.ctx, MACRO_PATHS[name]))

    def tuning_info(self):
        """Result of the sweep tile-shape autotuning of this solve."""
        return self.lib.gsis_tuning_info(self.ctx).decode()

    def hot(self):
        names = ["hot_sxx", "hot_syy", "hot_szz", "hot_sxy", "hot_sxz", "hot_syz", "hot_qx", "hot_qy", "hot_qz"]
        m = self.moments(names)
        return np.stack([m[n] for n in names], axis=1)

    def two_vdf_reference(self, S, d_r, Z_r, A):
        """Reference pair (g0, g1) of the two-VDF model (gsis_two_vdf_reference)
        for states S [n, 12] (rho, u (3), T_t, T_r, q_t (3), q_r (3)) on this
        solver's velocity grid; returns [n, 2, Nv] on the host."""
        import torch
        S = np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(-1, 12))
        n = S.shape[0]
        dS = torch.from_numpy(S).to("cuda")
        out = torch.empty((n, 2, self.nv), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()   # the library works on its own stream
        Ah = (ctypes.c_double * 4)(*[float(a) for a in A])
        self._check(self.lib.gsis_two_vdf_reference(self.ctx, ctypes.c_void_p(dS.data_ptr()), n, int(d_r),
                                                    float(Z_r), Ah, ctypes.c_void_p(out.data_ptr())))
        return out.cpu().numpy()

    def two_vdf_moments(self, F, d_r):
        """Moments of two-VDF pairs F [n, 2, Nv] on this solver's velocity grid
        (gsis_two_vdf_moments): [n, 18] = rho, u (3), T_t, T_r, sigma (6), q_t
        (3), q_r (3), on the host."""
        import torch
        F = np.ascontiguousarray(np.asarray(F, dtype=np.float64).reshape(-1, 2, self.nv))
        n = F.shape[0]
        dF = torch.from_numpy(F).to("cuda")
        out = torch.empty((n, 18), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()   # the library works on its own stream
        self._check(self.lib.gsis_two_vdf_moments(self.ctx, ctypes.c_void_p(dF.data_ptr()), n, int(d_r),
                                                  ctypes.c_void_p(out.data_ptr())))
        return out.cpu().numpy()

    def dvm_flags(self):
        return self.moments(("dvm",))["dvm"] > 0.5

    def vdf(self, n_dvm):
        out = np.zeros((n_dvm, self.nv))
        cells = np.zeros(max(n_dvm, 1), dtype=np.int32)
        self._check(self.lib.gsis_get_vdf(self.ctx, _dptr(out), cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                          out.size))
        return cells[:n_dvm], out

    def close(self):
        if self.ctx:
            self.lib.gsis_free(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ctx_array(solvers):
    arr = (ctypes.c_void_p * len(solvers))()
    for i, s in enumerate(solvers):
        arr[i] = s.ctx.value
    return arr


def iterate_batch(solvers, n):
    """Advance every solver by n GSIS iterations in one batched pass per
    iteration (gsis_iterate_batch); returns one report dict per solver."""
    lib = load()
    reps = (Report * len(solvers))()
    st = lib.gsis_iterate_batch(_ctx_array(solvers), len(solvers), int(n), reps)
    if st != GSIS_OK:
        msg = ""
        for s in solvers:
            e = lib.gsis_last_error(s.ctx)
            if e:
                msg = e.decode()
                break
        raise GsisError(st, msg)
    out = []
    for rep in reps:
        d = {f: getattr(rep, f) for f, _ in Report._fields_ if f != "phase_ms"}
        d["phase_ms"] = {PHASES[i]: rep.phase_ms[i] for i in range(8)}
        out.append(d)
    return out


def set_batch_tile(name):
    """Force the tile shape of batch plans recorded from now on (test hook);
    None or "" restores autotuning."""
    st = load().gsis_debug_set_batch_tile(name.encode() if name else None)
    if st != GSIS_OK:
        raise GsisError(st, "unknown batch tile %r" % name)


def batch_info(solvers):
    """Description of the recorded batch plan of this solver list."""
    return load().gsis_batch_info(_ctx_array(solvers), len(solvers)).decode()


def fma_peak(fp64, stream=None):
    """Measured FMA throughput of the current GPU's CUDA cores (flop/s) and
    the duration of the best timed launch (ms): FP64 if fp64 else FP32."""
    lib = load()
    r, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    st = lib.gsis_probe_fma_peak(1 if fp64 else 0, sp, ctypes.byref(r), ctypes.byref(ms))
    if st != GSIS_OK:
        raise GsisError(st, "FMA peak probe failed")
    return r.value, ms.value


def sweep_levels(neighbour_lists, key):
    """Sweep levels of an unstructured mesh (gsis_sweep_levels): neighbour_lists
    [ncell] of face-neighbour index lists, key [ncell]; returns (level [ncell],
    number of levels)."""
    lib = load()
    n = len(neighbour_lists)
    off = np.zeros(n + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(l) for l in neighbour_lists])
    nb = np.array([x for l in neighbour_lists for x in l] or [0], dtype=np.int32)
    k = np.ascontiguousarray(np.asarray(key, dtype=np.float64))
    lv = np.zeros(max(n, 1), dtype=np.int32)
    nl = ctypes.c_int(0)
    ip = ctypes.POINTER(ctypes.c_int)
    st = lib.gsis_sweep_levels(n, off.ctypes.data_as(ip), nb.ctypes.data_as(ip),
                               k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), lv.ctypes.data_as(ip),
                               ctypes.byref(nl))
    if st != GSIS_OK:
        raise GsisError(st, "invalid mesh adjacency or keys")
    return lv[:n].copy(), nl.value


def version():
    return load().gsis_version().decode()
