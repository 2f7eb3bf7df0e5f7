"""Thin ctypes binding of libhomelbm.so (C ABI in include/homelbm.h).

Only argument marshalling lives here: every step of the lattice update runs in
the library's CUDA kernels.  Host buffers are numpy arrays; device buffers are
torch CUDA tensors (passed by data pointer).  The binding raises if the library
is missing -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhomelbm.so")

OK, E_INVALID_ARG, E_BAD_STATE, E_OOM, E_CUDA, E_NONFINITE, E_TIMEOUT, E_UNSUPPORTED = range(8)
STORE_F64, STORE_F32, STORE_F16S, STORE_BF16S = range(4)
RESCALE_POST, RESCALE_PRE, RESCALE_PAPER = range(3)
STORAGE_NAMES = {"f64": STORE_F64, "f32": STORE_F32, "f16s": STORE_F16S, "bf16s": STORE_BF16S}
RESCALE_NAMES = {"post": RESCALE_POST, "pre": RESCALE_PRE, "paper": RESCALE_PAPER}
FLAG_LEAF, FLAG_BORDER, FLAG_NEW, FLAG_REFINE, FLAG_COARSEN = 1, 2, 4, 8, 16


class HlbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hlbm status %d: %s" % (code, msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("block_edge", ctypes.c_int32), ("num_levels", ctypes.c_int32),
        ("tau_finest", ctypes.c_double),
        ("periodic", ctypes.c_int32 * 3),
        ("storage", ctypes.c_int32), ("rescale_mode", ctypes.c_int32), ("xyz_literal", ctypes.c_int32),
        ("stream", ctypes.c_void_p), ("device", ctypes.c_int32),
    ]


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "hlbm_version": (ctypes.c_char_p, []),
    "hlbm_create": (ctypes.c_int32, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]),
    "hlbm_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "hlbm_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "hlbm_set_dense": (ctypes.c_int32, [ctypes.c_void_p]),
    "hlbm_set_fine_blocks": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "hlbm_set_blocks": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64]),
    "hlbm_rebuild_from_particles": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                     ctypes.c_int32, ctypes.c_void_p]),
    "hlbm_get_interface_nodes": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                                  ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "hlbm_num_blocks": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "hlbm_get_blocks": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]),
    "hlbm_set_uniform_force": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "hlbm_set_force": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "hlbm_set_solid": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p]),
    "hlbm_write_moments": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_int32]),
    "hlbm_read_moments": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32]),
    "hlbm_step": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "hlbm_synchronize": (ctypes.c_int32, [ctypes.c_void_p]),
    "hlbm_reduce": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "hlbm_forward_record": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]),
    "hlbm_inject_alloc_failure": (ctypes.c_int32, [ctypes.c_int64]),
    "hlbm_set_block_lookup": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "hlbm_set_profiling": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "hlbm_get_profile": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    "hlbm_get_block_lookup": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(ctypes.c_int64)]),
    "hlbm_test_narrow": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "hlbm_set_drag": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_int32]),
    "hlbm_set_open_faces": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int32]),
    "hlbm_adjoint": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "hlbm_reduce_f32_noalloc": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    "hlbm_deposit_particles": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_int64)]),
    "hlbm_batch_create": (ctypes.c_int32, [ctypes.POINTER(Config), ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "hlbm_batch_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "hlbm_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "hlbm_batch_num_blocks": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "hlbm_batch_write_moments": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                                  ctypes.c_int32]),
    "hlbm_batch_read_moments": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                                 ctypes.c_int32]),
    "hlbm_batch_step": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "hlbm_batch_synchronize": (ctypes.c_int32, [ctypes.c_void_p]),
    "hlbm_batch_set_mode": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "hlbm_batch_autotune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_float)]),
}
BATCH_ONE_LAUNCH, BATCH_GRAPH, BATCH_PER_DOMAIN, BATCH_PERSISTENT, BATCH_PERSISTENT_GRAPH = range(5)
FACE_CLOSED, FACE_OUTFLOW, FACE_INLET = range(3)


def exported_symbols():
    """Names of the C ABI entry points this binding expects."""
    return sorted(_SIGS)


def load(path=LIB_PATH):
    """Load libhomelbm.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libhomelbm.so not found at %s: run paper_2603_14982_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(buf):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(buf.ctypes.data), 0
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(buf.data_ptr()), 1 if buf.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def _f32(buf, what, device=False):
    """(pointer, on_device) of a float32 buffer the library reads as float32:
    any other dtype is refused rather than reinterpreted (a float64 tensor made
    under torch's default dtype would otherwise be read as pairs of floats)."""
    name = str(buf.dtype)
    if name not in ("float32", "torch.float32"):
        raise TypeError("%s must be float32, got %s" % (what, name))
    p, dev = _ptr(buf)
    if device and not dev:
        raise TypeError("%s must be a CUDA tensor" % what)
    return p, dev


def _dtype_code(buf):
    name = str(buf.dtype)
    if name in ("float64", "torch.float64"):
        return 0
    if name in ("float32", "torch.float32"):
        return 1
    raise TypeError("moment buffers must be float64 or float32, got %s" % name)


class Lattice:
    """One lattice handle (hlbm_lattice*)."""

    def __init__(self, extent, levels=1, tau=0.6, periodic=(True, True, True), storage="f32",
                 rescale="post", xyz_literal=False, stream=None, device=0):
        self.lib = load()
        cfg = Config()
        cfg.nx, cfg.ny, cfg.nz = (int(v) for v in extent)
        cfg.block_edge = 8
        cfg.num_levels = int(levels)
        cfg.tau_finest = float(tau)
        for a in range(3):
            cfg.periodic[a] = 1 if periodic[a] else 0
        cfg.storage = STORAGE_NAMES[storage] if isinstance(storage, str) else int(storage)
        cfg.rescale_mode = RESCALE_NAMES[rescale] if isinstance(rescale, str) else int(rescale)
        cfg.xyz_literal = 1 if xyz_literal else 0
        cfg.stream = ctypes.c_void_p(int(stream) if stream is not None else 0)
        cfg.device = int(device)
        self.cfg = cfg
        self.extent = tuple(int(v) for v in extent)
        self.levels = int(levels)
        h = ctypes.c_void_p()
        rc = self.lib.hlbm_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != OK:
            raise HlbmError(rc, self.lib.hlbm_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise HlbmError(rc, self.lib.hlbm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.hlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- blocks
    def set_dense(self):
        self._check(self.lib.hlbm_set_dense(self.h))

    def set_fine_blocks(self, coords):
        """coords: int32 (n, 3) level-0 block coordinates (bx, by, bz) where Phi = 0."""
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int32).reshape(-1, 3))
        self._check(self.lib.hlbm_set_fine_blocks(self.h, c.ctypes.data if len(c) else None, len(c)))

    def set_blocks(self, level, coords):
        """coords: int32 (n, 3) block coordinates (bx, by, bz) stored at `level`;
        the call that completes every level installs the hierarchy."""
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int32).reshape(-1, 3))
        self._check(self.lib.hlbm_set_blocks(self.h, int(level), c.ctypes.data if len(c) else None, len(c)))

    def rebuild_from_particles(self, pos):
        """pos: float32 (n, 3) numpy (host) or torch CUDA tensor; returns (refined, coarsened, deleted)."""
        counts = np.zeros(3, dtype=np.int64)
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float32)
        p, dev = _f32(pos, "particle positions")
        n = int(pos.shape[0])
        self._check(self.lib.hlbm_rebuild_from_particles(self.h, p if n else None, n, dev, counts.ctypes.data))
        return tuple(int(v) for v in counts)

    def set_block_lookup(self, mode):
        """0: dense per-level slot tables (default); 1: spatial hash per level."""
        self._check(self.lib.hlbm_set_block_lookup(self.h, int(mode)))

    PROFILE_CLASSES = ("stream_collide", "down", "up", "open_faces", "rebuild", "deposit", "adjoint", "reduce")

    def set_profiling(self, on=True):
        self._check(self.lib.hlbm_set_profiling(self.h, 1 if on else 0))

    def profile(self, reset=False):
        """{class: (ms of stream time, spans)} so far (synchronises)."""
        ms = (ctypes.c_double * 8)()
        cnt = (ctypes.c_int64 * 8)()
        self._check(self.lib.hlbm_get_profile(self.h, ms, cnt, 1 if reset else 0))
        return {name: (ms[i], cnt[i]) for i, name in enumerate(self.PROFILE_CLASSES)}

    def block_lookup(self):
        """(mode, device bytes of the lookup tables of all levels)."""
        mode, nbytes = ctypes.c_int32(), ctypes.c_int64()
        self._check(self.lib.hlbm_get_block_lookup(self.h, ctypes.byref(mode), ctypes.byref(nbytes)))
        return mode.value, nbytes.value

    def interface_nodes(self, level, which):
        """int32 array of (block << 9) | node of I^d (which=0) or I^u (which=1)."""
        n = ctypes.c_int64()
        self.lib.hlbm_get_interface_nodes(self.h, level, which, None, 0, ctypes.byref(n))
        out = np.zeros(max(n.value, 1), dtype=np.int32)
        self._check(self.lib.hlbm_get_interface_nodes(self.h, level, which, out.ctypes.data, n.value,
                                                      ctypes.byref(n)))
        return out[:n.value]

    def num_blocks(self, level=0):
        n = ctypes.c_int64()
        self._check(self.lib.hlbm_num_blocks(self.h, level, ctypes.byref(n)))
        return n.value

    def blocks(self, level=0):
        """(coords int32 (n, 3) as (bx, by, bz), flags uint8 (n,)) in slot order."""
        n = self.num_blocks(level)
        out = np.zeros((max(n, 1), 3), dtype=np.int32)
        fl = np.zeros(max(n, 1), dtype=np.uint8)
        nn = ctypes.c_int64()
        self._check(self.lib.hlbm_get_blocks(self.h, level, out.ctypes.data, n, ctypes.byref(nn), fl.ctypes.data))
        return out[:n], fl[:n]

    # ---- inputs
    def deposit_particles(self, pos, kappa=1e-4, eta_max=0.4, per_particle=0.25, moving=True, wait=True):
        """Finest-level eta / eps / drag force from particle positions (float32 [n][3],
        numpy or CUDA tensor).  wait=True returns the number of particles dropped;
        wait=False returns None without waiting for the stream."""
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float32)
        p, dev = _f32(pos, "particle positions")
        out = ctypes.c_int64()
        self._check(self.lib.hlbm_deposit_particles(self.h, p, int(pos.shape[0]), dev, float(kappa), float(eta_max),
                                                    float(per_particle), 1 if moving else 0,
                                                    ctypes.byref(out) if wait else None))
        return out.value if wait else None

    def set_uniform_force(self, fx, fy, fz):
        self._check(self.lib.hlbm_set_uniform_force(self.h, float(fx), float(fy), float(fz)))

    def set_force(self, F=None, eps=None):
        """F: torch CUDA float32 [n0][3][512] (or None), eps: [n0][512] (or None)."""
        pF = _f32(F, "F", device=True)[0] if F is not None else None
        pe = _f32(eps, "eps", device=True)[0] if eps is not None else None
        self._check(self.lib.hlbm_set_force(self.h, pF, pe))

    def set_drag(self, kappa, vp, exchange_every):
        """Live drag F = kappa (1 - eps) (vp - u*) exchanged every ``exchange_every``
        level-0 steps (0 = off); see hlbm_set_drag."""
        v = (ctypes.c_double * 3)(*(float(x) for x in vp))
        self._check(self.lib.hlbm_set_drag(self.h, float(kappa), v, int(exchange_every)))

    def set_open_faces(self, types, u0=0.0, beta=0.0, h0=0.0, profile_axis=1):
        """types: 6 face conditions (x-, x+, y-, y+, z-, z+) from FACE_*; see hlbm_set_open_faces."""
        t = (ctypes.c_int32 * 6)(*(int(v) for v in types))
        self._check(self.lib.hlbm_set_open_faces(self.h, t, float(u0), float(beta), float(h0), int(profile_axis)))

    def set_solid(self, mask_dense):
        """mask_dense: numpy uint8/bool [nz][ny][nx] (fine nodes), or None."""
        if mask_dense is None:
            self._check(self.lib.hlbm_set_solid(self.h, None))
            return
        m = np.ascontiguousarray(mask_dense, dtype=np.uint8)
        self._check(self.lib.hlbm_set_solid(self.h, m.ctypes.data))

    # ---- moments
    def write_moments(self, buf, level=0):
        p, dev = _ptr(buf)
        self._check(self.lib.hlbm_write_moments(self.h, level, p, _dtype_code(buf), dev))

    def read_moments(self, buf=None, level=0, physical_u=False, dtype=np.float64):
        """Fill ``buf`` (numpy host array or torch CUDA tensor, [n][10][512]) and return it."""
        if buf is None:
            buf = np.empty((self.num_blocks(level), 10, 512), dtype=dtype)
        p, dev = _ptr(buf)
        self._check(self.lib.hlbm_read_moments(self.h, level, p, _dtype_code(buf), dev, 1 if physical_u else 0))
        return buf

    # ---- stepping
    def step(self, n_fine_steps=1):
        self._check(self.lib.hlbm_step(self.h, int(n_fine_steps)))

    def forward_record(self, n_steps, ckpt_every):
        self._check(self.lib.hlbm_forward_record(self.h, int(n_steps), int(ckpt_every)))

    def adjoint(self, dL_dM, dL_dF):
        """dL_dM: torch CUDA float32 [n][10][512] of the final state (multi-level
        lattices: every level's blocks, level 0 first); dL_dF: torch CUDA
        float32 [n0][3][512] (written)."""
        self._check(self.lib.hlbm_adjoint(self.h, _f32(dL_dM, "dL_dM", device=True)[0],
                                          _f32(dL_dF, "dL_dF", device=True)[0]))
        return dL_dF

    def synchronize(self):
        self._check(self.lib.hlbm_synchronize(self.h))

    def reduce(self):
        out = (ctypes.c_double * 7)()
        self._check(self.lib.hlbm_reduce(self.h, out))
        return np.array(out[:], dtype=np.float64)


class Batch:
    """A batch of independent single-level periodic domains (hlbm_batch*).

    ``domains`` is a list of ((nx, ny, nz), tau) pairs."""

    def __init__(self, domains, storage="f16s", xyz_literal=False, stream=None, device=0):
        self.lib = load()
        n = len(domains)
        cfgs = (Config * n)()
        for c, (extent, tau) in zip(cfgs, domains):
            c.nx, c.ny, c.nz = (int(v) for v in extent)
            c.block_edge = 8
            c.num_levels = 1
            c.tau_finest = float(tau)
            for a in range(3):
                c.periodic[a] = 1
            c.storage = STORAGE_NAMES[storage] if isinstance(storage, str) else int(storage)
            c.rescale_mode = RESCALE_POST
            c.xyz_literal = 1 if xyz_literal else 0
            c.stream = ctypes.c_void_p(int(stream) if stream is not None else 0)
            c.device = int(device)
        self.domains = [(tuple(int(v) for v in e), float(t)) for e, t in domains]
        h = ctypes.c_void_p()
        rc = self.lib.hlbm_batch_create(cfgs, n, ctypes.byref(h))
        if rc != OK:
            raise HlbmError(rc, self.lib.hlbm_batch_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise HlbmError(rc, self.lib.hlbm_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.hlbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def num_blocks(self, domain=-1):
        n = ctypes.c_int64()
        self._check(self.lib.hlbm_batch_num_blocks(self.h, int(domain), ctypes.byref(n)))
        return n.value

    def write_moments(self, domain, buf):
        p, dev = _ptr(buf)
        self._check(self.lib.hlbm_batch_write_moments(self.h, int(domain), p, _dtype_code(buf), dev))

    def read_moments(self, domain, buf=None, dtype=np.float64):
        if buf is None:
            buf = np.empty((self.num_blocks(domain), 10, 512), dtype=dtype)
        p, dev = _ptr(buf)
        self._check(self.lib.hlbm_batch_read_moments(self.h, int(domain), p, _dtype_code(buf), dev))
        return buf

    def step(self, n_steps=1):
        self._check(self.lib.hlbm_batch_step(self.h, int(n_steps)))

    def synchronize(self):
        self._check(self.lib.hlbm_batch_synchronize(self.h))

    def set_mode(self, mode):
        self._check(self.lib.hlbm_batch_set_mode(self.h, int(mode)))

    def autotune(self, trial_steps=64):
        mode = ctypes.c_int32()
        ms = (ctypes.c_float * 5)()
        self._check(self.lib.hlbm_batch_autotune(self.h, int(trial_steps), ctypes.byref(mode), ms))
        return mode.value, [float(v) for v in ms]


# ---- layout marshalling between dense [10][nz][ny][nx] grids and block-major [n][10][512]

def dense_to_blocks(M, coords=None):
    """Dense (R, nz, ny, nx) -> block-major (n, R, 512) for the given block coords
    (default: every block in slot order)."""
    M = np.asarray(M)
    R, nz, ny, nx = M.shape
    t = M.reshape(R, nz // 8, 8, ny // 8, 8, nx // 8, 8).transpose(1, 3, 5, 0, 2, 4, 6)
    t = t.reshape(nz // 8, ny // 8, nx // 8, R, 512)
    if coords is None:
        return np.ascontiguousarray(t.reshape(-1, R, 512))
    c = np.asarray(coords)
    return np.ascontiguousarray(t[c[:, 2], c[:, 1], c[:, 0]])


def blocks_to_dense(Mb, shape, coords=None, fill=np.nan):
    """Block-major (n, R, 512) -> dense (R, nz, ny, nx); nodes of absent blocks hold ``fill``."""
    Mb = np.asarray(Mb)
    nz, ny, nx = shape
    R = Mb.shape[1]
    t = np.full((nz // 8, ny // 8, nx // 8, R, 512), fill, dtype=Mb.dtype)
    if coords is None:
        t = Mb.reshape(nz // 8, ny // 8, nx // 8, R, 512)
    else:
        c = np.asarray(coords)
        t[c[:, 2], c[:, 1], c[:, 0]] = Mb
    t = t.reshape(nz // 8, ny // 8, nx // 8, R, 8, 8, 8).transpose(3, 0, 4, 1, 5, 2, 6)
    return np.ascontiguousarray(t.reshape(R, nz, ny, nx))


def inject_alloc_failure(after):
    """Test hook: the device allocation after ``after`` more successful ones
    fails with E_OOM (after < 0 clears); see hlbm_inject_alloc_failure."""
    load().hlbm_inject_alloc_failure(int(after))


def make_force_autograd(lattice, n_steps, ckpt_every):
    """A torch.autograd.Function mapping the level-0 force field F ([n0][3][512]
    float32 CUDA) to the stored moments after ``n_steps`` fine steps from the
    lattice's current state ([n][10][512] float32 CUDA, public layout; every
    level's blocks, level 0 first).  The backward pass runs the library's
    checkpointed adjoint."""
    import torch

    class ForceToMoments(torch.autograd.Function):
        @staticmethod
        def forward(ctx, F):
            Fc = F.detach().contiguous()
            lattice.set_force(Fc)
            lattice.forward_record(n_steps, ckpt_every)
            counts = [lattice.num_blocks(l) for l in range(lattice.levels)]
            out = torch.empty((sum(counts), 10, 512), dtype=torch.float32, device=F.device)
            o = 0
            for l, n in enumerate(counts):
                if n:
                    lattice.read_moments(out[o:o + n], level=l)
                o += n
            lattice.synchronize()
            return out

        @staticmethod
        def backward(ctx, grad_out):
            dF = torch.empty((lattice.num_blocks(0), 3, 512), dtype=torch.float32, device=grad_out.device)
            lattice.adjoint(grad_out.contiguous().float(), dF)
            return dF

    return ForceToMoments.apply
