"""Python binding of the GB300 NFS structure-function library (include/nfs.h).

Argument marshalling only: every step of the analysis (mean normalisation, FFTs, the delay update
of Eq. 1, radial binning) runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing, importing works but constructing ``NFS`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "_build", "libnfs_gb300.so")
HEADER = os.path.join(ROOT, "include", "nfs.h")

NFS_OK = 0
NFS_EINVAL = -1
NFS_EUNSUPPORTED = -2
NFS_ENOMEM = -3
NFS_ECUDA = -4
NFS_ESTATE = -5
NFS_ETOOBIG = -6
NFS_ETIMEOUT = -7
NOALLOC_SCRATCH_BYTES = 64 << 20
PATH_FUSED_F32 = 0
PATH_PLAIN_F64 = 1
OPT_TIMING = 1
OPT_BLOCK_FRAMES = 2
OPT_RING_SLOTS = 3
OPT_PITCH = 4
OPT_PATH = 5
OPT_FFT_CHUNK = 6
OPT_DELAY_VARIANT = 7
OPT_FFT_GENERIC = 8
OPT_TEST_STALL_GROUP = 9
OPT_SLAB_FIRST_MODE = 10
OPT_SLAB_MODES = 11
OPT_DELAY_SPAN = 12
OPT_H2D = 13
OPT_MODES = 14
OPT_DELAY_MODES = 15
FIT_GAUSS_NEWTON = 0
FIT_ADAM = 1
STAGES = ("h2d", "mean", "rowfft", "colfft", "delay", "bin")

_lib = None


class NFSError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_text(status)} ({status}){': ' + detail if detail else ''}")


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def load_library(path: Optional[str] = None):
    """Load libnfs_gb300.so and declare its signatures (raises if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(p)
    V, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "nfs_create": (I, [I, I, V, I, I, PP]),
        "nfs_create_ex": (I, [I, I, V, I, I, I, I, PP]),
        "nfs_create_slab": (I, [I, I, V, I, I, I, I, PP]),
        "nfs_slab_range": (I, [I, I, I, I, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "nfs_push_frames": (I, [V, V, I]),
        "nfs_push_frames_device": (I, [V, V, I]),
        "nfs_structure_function": (I, [V, V, V, V, V]),
        "nfs_export_spectrum": (I, [V, I, V]),
        "nfs_reset": (I, [V]),
        "nfs_synchronize": (I, [V]),
        "nfs_frame_count": (I64, [V]),
        "nfs_destroy": (None, [V]),
        "nfs_strerror": (ctypes.c_char_p, [I]),
        "nfs_last_error": (ctypes.c_char_p, [V]),
        "nfs_get_stream": (V, [V]),
        "nfs_set_option": (I, [V, I, I64]),
        "nfs_get_option": (I, [V, I, ctypes.POINTER(I64)]),
        "nfs_get_timings": (I, [V, V, V]),
        "nfs_reset_timings": (I, [V]),
        "nfs_get_timeline": (I, [V, V, V, V, I64, ctypes.POINTER(I64)]),
        "nfs_launch_count": (I64, [V]),
        "nfs_delay_profile": (I, [V, I, I]),
        "nfs_structure_function_noalloc": (I, [V, I, I, I, V, I, I, V, V, V, V]),
        "nfs_out_of_core_plan": (I, [V, I, I64, I64, V, V, ctypes.POINTER(I), ctypes.POINTER(I64)]),
        "nfs_delay_schedule": (I, [V, I, I, V, V, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                   ctypes.POINTER(I), ctypes.POINTER(I), I]),
        "nfs_structure_function_out_of_core": (I, [I, I, V, I, I, V, I64, I64, V, V, V, V, ctypes.POINTER(I64)]),
        "nfs_fit": (I, [V, V, V, V, V, I, I]),
        "nfs_batch_create": (I, [I, V, V, V, V, V, PP]),
        "nfs_batch_destroy": (None, [V]),
        "nfs_batch_push": (I, [V, I, V, I]),
        "nfs_batch_push_device": (I, [V, V, V]),
        "nfs_batch_structure_function": (I, [V, I, V, V, V, V]),
        "nfs_batch_reset": (I, [V]),
        "nfs_batch_synchronize": (I, [V]),
        "nfs_batch_member": (V, [V, I]),
        "nfs_batch_get_stream": (V, [V]),
        "nfs_batch_launch_count": (I64, [V]),
        "nfs_batch_last_error": (ctypes.c_char_p, [V]),
        "nfs_roi_create": (I, [I, I, I, V, V, V, V, V, I, V, PP]),
        "nfs_bin_table": (I, [I, I, I, V, V, V]),
        "nfs_roi_push": (I, [V, V, I]),
        "nfs_roi_push_device": (I, [V, V, I]),
        "nfs_fit_loss_grad": (I, [V, V, I, I, V, V, V, V, V, V, V, V]),
        "nfs_fit_gauss_newton": (I, [V, V, I, I, V, V, V, I, ctypes.c_float, V]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = L
    return L


def header_functions(header: str = HEADER):
    """Names of the functions declared in the public header."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nfs_[a-z0-9_]+)\s*\(", text)))


def status_text(status: int) -> str:
    try:
        return load_library().nfs_strerror(status).decode()
    except Exception:
        return {0: "ok", -1: "invalid argument", -2: "unsupported frame shape", -3: "out of memory",
                -4: "CUDA error", -5: "call not allowed in this state",
                -6: "problem too large for the no-allocation scratch", -7: "a device-side wait ran out of time"}.get(status, "unknown status")


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _after_current_stream(stream_handle: int, device):
    """Make the library's stream wait for the work queued so far on PyTorch's current stream (which
    may still be writing the frames about to be pushed)."""
    import torch
    ev = torch.cuda.Event()
    ev.record(torch.cuda.current_stream(device))
    torch.cuda.ExternalStream(stream_handle, device=device).wait_event(ev)


class _InFlight:
    """Device tensors the library may still be reading on its own stream, each with an event
    recorded on that stream after its push: the tensors stay referenced (so PyTorch's caching
    allocator cannot hand their memory to other tensors) until their events have completed; entries
    are dropped as they complete and all at once after calls that synchronise the stream.  (The C
    ABI requires device frames to stay valid until the context's stream has passed them.)"""

    def __init__(self):
        self.items = []

    def add(self, tensor, stream_handle: int):
        import torch
        ev = torch.cuda.Event()
        ev.record(torch.cuda.ExternalStream(stream_handle, device=tensor.device))
        self.items = [(t, e) for (t, e) in self.items if not e.query()]
        self.items.append((tensor, ev))

    def clear(self):
        self.items = []


class NFS:
    """One analysis context: frames in, binned structure function D_b(tau) out (Eq. 1, Fig. 1e,f)."""

    def __init__(self, H: int, W: int, delays: Sequence[int], n_qbins: int, path: str = "f32",
                 block_frames: int = 0, slab: int = 0, n_slabs: int = 1):
        """slab, n_slabs: keep only that share of the modes (nfs_create_slab; the D of all slabs of
        one frame sequence add up to the whole D, see reduce_slabs)."""
        self._L = load_library()
        self.H, self.W = int(H), int(W)
        self.delays = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
        self.n_qbins = int(n_qbins)
        self.path = {"f32": PATH_FUSED_F32, "f64": PATH_PLAIN_F64}[path]
        h = ctypes.c_void_p()
        if n_slabs != 1:
            if self.path != PATH_FUSED_F32 or block_frames:
                raise ValueError("mode slabs run on the fused FP32 path with the default block")
            rc = self._L.nfs_create_slab(self.H, self.W, _ptr(self.delays), int(self.delays.size), self.n_qbins,
                                         int(slab), int(n_slabs), ctypes.byref(h))
            what = "nfs_create_slab"
        else:
            rc = self._L.nfs_create_ex(self.H, self.W, _ptr(self.delays), int(self.delays.size), self.n_qbins,
                                       self.path, int(block_frames), ctypes.byref(h))
            what = "nfs_create_ex"
        if rc != NFS_OK:
            raise NFSError(rc, what)
        self._h = h
        self._inflight = _InFlight()

    # --------------------------------------------------------------- helpers
    def _check(self, rc: int, what: str):
        if rc != NFS_OK:
            detail = self._L.nfs_last_error(self._h) if self._h else b""
            raise NFSError(rc, what, (detail or b"").decode())

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._L.nfs_destroy(self._h)  # synchronises the context's streams first
            self._h = None
        if getattr(self, "_inflight", None):
            self._inflight.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --------------------------------------------------------------- frames
    def push_frames(self, frames) -> None:
        """Host frames [n, H, W] uint16 (numpy, or a CPU torch tensor, pinned or not)."""
        if hasattr(frames, "data_ptr"):
            t = frames
            assert not t.is_cuda and t.is_contiguous() and t.element_size() == 2
            n = t.shape[0] if t.dim() == 3 else 1
            self._check(self._L.nfs_push_frames(self._h, ctypes.c_void_p(t.data_ptr()), n), "nfs_push_frames")
            return
        a = np.ascontiguousarray(frames, dtype=np.uint16)
        if a.ndim == 2:
            a = a[None]
        assert a.shape[1:] == (self.H, self.W), a.shape
        self._check(self._L.nfs_push_frames(self._h, _ptr(a), a.shape[0]), "nfs_push_frames")

    def push_frames_device(self, frames) -> None:
        """Device frames: a CUDA torch tensor [n, H, W] of 2-byte integers (int16 storage of counts).

        The library reads them asynchronously on its own stream: that stream first waits for the
        work already queued on PyTorch's current stream (which may still be writing the frames), and
        the context keeps the tensor referenced until its stream has read it, so PyTorch does not
        hand its memory to other tensors even if the caller drops it at once."""
        assert frames.is_cuda and frames.is_contiguous() and frames.element_size() == 2
        n = frames.shape[0] if frames.dim() == 3 else 1
        _after_current_stream(self.stream, frames.device)
        self._check(self._L.nfs_push_frames_device(self._h, ctypes.c_void_p(frames.data_ptr()), n),
                    "nfs_push_frames_device")
        self._inflight.add(frames, self.stream)

    def push_frames_device_ptr(self, ptr: int, n: int) -> None:
        self._check(self._L.nfs_push_frames_device(self._h, ctypes.c_void_p(ptr), int(n)), "nfs_push_frames_device")

    # --------------------------------------------------------------- results
    def structure_function(self) -> dict:
        nd, nq = self.delays.size, self.n_qbins
        D = np.zeros((nd, nq), np.float64)
        bc = np.zeros(nq, np.int64)
        pc = np.zeros(nd, np.int64)
        qm = np.zeros(nq, np.float64)
        self._check(self._L.nfs_structure_function(self._h, _ptr(D), _ptr(bc), _ptr(pc), _ptr(qm)),
                    "nfs_structure_function")
        self._inflight.clear()  # the call synchronised the stream
        return dict(D=D, bin_counts=bc, pair_counts=pc, q_mean=qm)

    def export_spectrum(self, j: int) -> np.ndarray:
        out = np.zeros((self.H, self.W // 2 + 1), np.float64)
        self._check(self._L.nfs_export_spectrum(self._h, int(j), _ptr(out)), "nfs_export_spectrum")
        return out

    def reset(self):
        self._check(self._L.nfs_reset(self._h), "nfs_reset")

    def synchronize(self):
        self._check(self._L.nfs_synchronize(self._h), "nfs_synchronize")
        self._inflight.clear()

    @property
    def frame_count(self) -> int:
        return int(self._L.nfs_frame_count(self._h))

    @property
    def stream(self) -> int:
        return int(self._L.nfs_get_stream(self._h) or 0)

    @property
    def launch_count(self) -> int:
        return int(self._L.nfs_launch_count(self._h))

    def set_option(self, key: int, value: int):
        self._check(self._L.nfs_set_option(self._h, int(key), int(value)), "nfs_set_option")

    def get_option(self, key: int) -> int:
        v = ctypes.c_int64()
        self._check(self._L.nfs_get_option(self._h, int(key), ctypes.byref(v)), "nfs_get_option")
        return int(v.value)

    def timings(self) -> dict:
        ms = np.zeros(len(STAGES), np.float64)
        n = np.zeros(len(STAGES), np.int64)
        self._check(self._L.nfs_get_timings(self._h, _ptr(ms), _ptr(n)), "nfs_get_timings")
        return {s: (float(ms[i]), int(n[i])) for i, s in enumerate(STAGES)}

    def reset_timings(self):
        self._check(self._L.nfs_reset_timings(self._h), "nfs_reset_timings")

    def timeline(self) -> list:
        """[(stage name, start ms, end ms)] of every launch and copy since reset_timings (needs
        set_option(OPT_TIMING, 3)); times from the first recorded launch."""
        n = ctypes.c_int64(0)
        self._check(self._L.nfs_get_timeline(self._h, None, None, None, 0, ctypes.byref(n)), "nfs_get_timeline")
        m = n.value
        st = np.zeros(max(m, 1), np.int32)
        a = np.zeros(max(m, 1), np.float64)
        e = np.zeros(max(m, 1), np.float64)
        self._check(self._L.nfs_get_timeline(self._h, _ptr(st), _ptr(a), _ptr(e), m, ctypes.byref(n)),
                    "nfs_get_timeline")
        return [(STAGES[int(st[i])], float(a[i]), float(e[i])) for i in range(m)]

    def fit(self, A, B, Gamma, iters: int = 50, method: int = FIT_GAUSS_NEWTON, D=None):
        """Fit Eq. 1 per bin (nfs_fit); initial A, B, Gamma in, fitted arrays returned."""
        nq = self.n_qbins
        a = np.ascontiguousarray(np.asarray(A, np.float32).reshape(nq)).copy()
        b = np.ascontiguousarray(np.asarray(B, np.float32).reshape(nq)).copy()
        g = np.ascontiguousarray(np.asarray(Gamma, np.float32).reshape(nq)).copy()
        d = None if D is None else np.ascontiguousarray(np.asarray(D, np.float64))
        self._check(self._L.nfs_fit(self._h, _ptr(d), _ptr(a), _ptr(b), _ptr(g), int(iters), int(method)), "nfs_fit")
        return a, b, g


def slab_range(H: int, W: int, slab: int, n_slabs: int):
    """(first mode, modes) of a slab in the column-major order k = k_x H + k_y (host logic)."""
    L = load_library()
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = L.nfs_slab_range(int(H), int(W), int(slab), int(n_slabs), ctypes.byref(a), ctypes.byref(b))
    if rc != NFS_OK:
        raise NFSError(rc, "nfs_slab_range")
    return a.value, b.value


def reduce_slabs(results, group=None) -> dict:
    """The whole result from the structure functions of the slabs of one frame sequence: D summed
    (each slab's D is its share of every bin average); counts and q_mean are the slabs' common ones.

    results: a list of per-slab dicts (slabs in one process), or, with a torch.distributed process
    group, this rank's own dict: D is then summed over the group's ranks (one all-reduce of
    n_delays x n_qbins doubles, in host memory: use a gloo group)."""
    if group is None:
        out = dict(results[0])
        D = np.zeros_like(results[0]["D"])
        for r in results:
            assert np.array_equal(r["bin_counts"], out["bin_counts"]) and np.array_equal(r["pair_counts"],
                                                                                          out["pair_counts"])
            D = D + r["D"]
        out["D"] = D
        return out
    import torch
    import torch.distributed as dist
    out = dict(results)
    t = torch.from_numpy(np.ascontiguousarray(out["D"], dtype=np.float64).copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    out["D"] = t.numpy()
    return out


def structure_function_noalloc(frames, delays, n_qbins: int, stream: int = 0) -> dict:
    """One-shot analysis of device frames that allocates no device memory (its scratch is a fixed
    static array in the library; see nfs_structure_function_noalloc in include/nfs.h).

    frames: CUDA tensor [n, H, W] of 2-byte integers.  Calls on one device must not overlap.
    """
    import torch
    L = load_library()
    assert frames.is_cuda and frames.is_contiguous() and frames.element_size() == 2 and frames.dim() == 3
    n, H, W = frames.shape
    d = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
    D = np.zeros((d.size, int(n_qbins)), np.float64)
    bc = np.zeros(int(n_qbins), np.int64)
    pc = np.zeros(d.size, np.int64)
    with torch.cuda.device(frames.device):  # the call runs on the current device: the frames' own
        rc = L.nfs_structure_function_noalloc(ctypes.c_void_p(frames.data_ptr()), int(n), int(H), int(W), _ptr(d),
                                              int(d.size), int(n_qbins), ctypes.c_void_p(stream or None), _ptr(D),
                                              _ptr(bc), _ptr(pc))
    if rc != NFS_OK:
        raise NFSError(rc, "nfs_structure_function_noalloc")
    return dict(D=D, bin_counts=bc, pair_counts=pc)


def bin_table(H: int, W: int, n_qbins: int) -> dict:
    """The radial bin table (nfs_bin_table): bin_of_mode [H][W/2+1] (-1 = excluded), bin_counts,
    q_mean.  Host computation only."""
    L = load_library()
    b = np.empty((int(H), int(W) // 2 + 1), np.int32)
    c = np.empty(int(n_qbins), np.int64)
    q = np.empty(int(n_qbins), np.float64)
    rc = L.nfs_bin_table(int(H), int(W), int(n_qbins), _ptr(b), _ptr(c), _ptr(q))
    if rc != NFS_OK:
        raise NFSError(rc, "nfs_bin_table")
    return dict(bin_of_mode=b, bin_counts=c, q_mean=q)


def out_of_core_plan(delays, n_frames: int, max_ring_slots: int) -> dict:
    """Bands of the out-of-core mode (host logic only; see nfs_out_of_core_plan)."""
    L = load_library()
    d = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
    first = np.zeros(d.size + 1, np.int32)
    shift = np.zeros(d.size, np.int64)
    nb = ctypes.c_int(0)
    nt = ctypes.c_int64(0)
    rc = L.nfs_out_of_core_plan(_ptr(d), int(d.size), int(n_frames), int(max_ring_slots), _ptr(first), _ptr(shift),
                                ctypes.byref(nb), ctypes.byref(nt))
    if rc != NFS_OK:
        raise NFSError(rc, "nfs_out_of_core_plan")
    n = nb.value
    return dict(band_first=first[:n + 1].copy(), band_shift=shift[:n].copy(), n_transforms=nt.value)


def delay_schedule(delays, cross: bool = False, span: int = 0) -> dict:
    """The fused delay kernel's copy schedule for a delay list (host logic; see nfs_delay_schedule;
    span 0 = the default)."""
    L = load_library()
    d = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
    cap = max(16, d.size)
    sr = np.zeros((cap, 3), np.int32)
    st = np.zeros((cap, 5), np.int32)
    out = [ctypes.c_int(0) for _ in range(5)]
    rc = L.nfs_delay_schedule(_ptr(d), int(d.size), int(bool(cross)), _ptr(sr), _ptr(st), cap,
                              *[ctypes.byref(o) for o in out], int(span))
    if rc != NFS_OK:
        raise NFSError(rc, "nfs_delay_schedule")
    nsr, nst, K, rows, bars = (o.value for o in out)
    return dict(subruns=sr[:nsr].copy(), stages=st[:nst].copy(), block_frames=K, slot_rows=rows, copy_barriers=bars)


def structure_function_out_of_core(frames, delays, n_qbins: int, max_ring_slots: int) -> dict:
    """Binned D of host frames [N, H, W] uint16 with at most max_ring_slots spectra on the device
    (bands of delays, each a pass over the frames; see nfs_structure_function_out_of_core)."""
    L = load_library()
    a = np.ascontiguousarray(frames.numpy() if hasattr(frames, "numpy") else frames)
    a = a.view(np.uint16) if a.dtype == np.int16 else a.astype(np.uint16, copy=False)
    N, H, W = a.shape
    d = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
    D = np.zeros((d.size, int(n_qbins)), np.float64)
    bc = np.zeros(int(n_qbins), np.int64)
    pc = np.zeros(d.size, np.int64)
    qm = np.zeros(int(n_qbins), np.float64)
    nt = ctypes.c_int64(0)
    rc = L.nfs_structure_function_out_of_core(int(H), int(W), _ptr(d), int(d.size), int(n_qbins), _ptr(a), int(N),
                                              int(max_ring_slots), _ptr(D), _ptr(bc), _ptr(pc), _ptr(qm),
                                              ctypes.byref(nt))
    if rc != NFS_OK:
        raise NFSError(rc, "nfs_structure_function_out_of_core")
    return dict(D=D, bin_counts=bc, pair_counts=pc, q_mean=qm, n_transforms=nt.value)


class NFSBatch:
    """Ragged batch of sequences (nfs_batch_*): uneven frame shapes and delay lists, one persistent
    delay-update launch per frame block for all members."""

    def __init__(self, shapes, delays_per_seq, n_qbins):
        self._L = load_library()
        self.shapes = [(int(h), int(w)) for h, w in shapes]
        n = len(self.shapes)
        self.delays = [np.ascontiguousarray(np.asarray(d, np.int32)) for d in delays_per_seq]
        self.n_qbins = [int(q) for q in n_qbins]
        assert len(self.delays) == n and len(self.n_qbins) == n
        H = np.array([h for h, _ in self.shapes], np.int32)
        W = np.array([w for _, w in self.shapes], np.int32)
        off = np.zeros(n + 1, np.int32)
        off[1:] = np.cumsum([d.size for d in self.delays])
        flat = np.ascontiguousarray(np.concatenate(self.delays).astype(np.int32))
        nq = np.array(self.n_qbins, np.int32)
        h = ctypes.c_void_p()
        rc = self._L.nfs_batch_create(n, _ptr(H), _ptr(W), _ptr(off), _ptr(flat), _ptr(nq), ctypes.byref(h))
        if rc != NFS_OK:
            raise NFSError(rc, "nfs_batch_create")
        self._h = h
        self._inflight = _InFlight()

    def _check(self, rc, what):
        if rc != NFS_OK:
            raise NFSError(rc, what, (self._L.nfs_batch_last_error(self._h) or b"").decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.nfs_batch_destroy(self._h)
            self._h = None
        if getattr(self, "_inflight", None):
            self._inflight.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def push_frames(self, seq, frames):
        a = np.ascontiguousarray(frames, dtype=np.uint16)
        self._check(self._L.nfs_batch_push(self._h, int(seq), _ptr(a), a.shape[0]), "nfs_batch_push")

    def push_frames_device(self, tensors):
        """tensors[s]: CUDA tensor [n_s, H_s, W_s] of 2-byte integers (or None for no frames)."""
        n = len(self.shapes)
        ptrs = (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in tensors])
        counts = np.array([(t.shape[0] if t is not None else 0) for t in tensors], np.int32)
        dev = next((t.device for t in tensors if t is not None), None)
        if dev is not None:
            _after_current_stream(self.stream, dev)
        self._check(self._L.nfs_batch_push_device(self._h, ptrs, _ptr(counts)), "nfs_batch_push_device")
        for t in tensors:
            if t is not None:
                self._inflight.add(t, self.stream)

    def structure_function(self, seq):
        nd, nq = self.delays[seq].size, self.n_qbins[seq]
        D = np.zeros((nd, nq), np.float64)
        bc = np.zeros(nq, np.int64)
        pc = np.zeros(nd, np.int64)
        qm = np.zeros(nq, np.float64)
        self._check(self._L.nfs_batch_structure_function(self._h, int(seq), _ptr(D), _ptr(bc), _ptr(pc), _ptr(qm)),
                    "nfs_batch_structure_function")
        self._inflight.clear()  # the call synchronised the batch's stream
        return dict(D=D, bin_counts=bc, pair_counts=pc, q_mean=qm)

    def reset(self):
        self._check(self._L.nfs_batch_reset(self._h), "nfs_batch_reset")

    def synchronize(self):
        self._check(self._L.nfs_batch_synchronize(self._h), "nfs_batch_synchronize")
        self._inflight.clear()

    @property
    def stream(self) -> int:
        return int(self._L.nfs_batch_get_stream(self._h) or 0)

    @property
    def launch_count(self) -> int:
        return int(self._L.nfs_batch_launch_count(self._h))

    def member_option(self, seq, key) -> int:
        v = ctypes.c_int64()
        c = self._L.nfs_batch_member(self._h, int(seq))
        rc = self._L.nfs_get_option(c, int(key), ctypes.byref(v))
        if rc != NFS_OK:
            raise NFSError(rc, "nfs_get_option")
        return int(v.value)


class NFSRoi(NFSBatch):
    """Regions of interest of one camera sequence (nfs_roi_*): window r = (y0, x0, h, w) of every
    H x W frame is analysed as a sequence of its own; structure_function(r) gives its result."""

    def __init__(self, H, W, rois, delays, n_qbins):
        self._L = load_library()
        self.H, self.W = int(H), int(W)
        self.rois = [tuple(int(v) for v in r) for r in rois]
        n = len(self.rois)
        self.shapes = [(h, w) for _, _, h, w in self.rois]
        d = np.ascontiguousarray(np.asarray(delays, np.int32))
        self.delays = [d] * n
        self.n_qbins = [int(q) for q in (n_qbins if np.ndim(n_qbins) else [n_qbins] * n)]
        assert len(self.n_qbins) == n
        y0, x0, h, w = (np.array([r[i] for r in self.rois], np.int32) for i in range(4))
        nq = np.array(self.n_qbins, np.int32)
        hdl = ctypes.c_void_p()
        rc = self._L.nfs_roi_create(self.H, self.W, n, _ptr(y0), _ptr(x0), _ptr(h), _ptr(w), _ptr(d), d.size,
                                    _ptr(nq), ctypes.byref(hdl))
        if rc != NFS_OK:
            raise NFSError(rc, "nfs_roi_create")
        self._h = hdl
        self._inflight = _InFlight()

    def push_frames(self, frames):
        """frames: [n, H, W] full frames in host memory (numpy, or a CPU torch tensor, pinned or not)."""
        if hasattr(frames, "data_ptr"):
            t = frames
            assert not t.is_cuda and t.is_contiguous() and t.element_size() == 2
            assert tuple(t.shape[1:]) == (self.H, self.W)
            self._check(self._L.nfs_roi_push(self._h, ctypes.c_void_p(t.data_ptr()), t.shape[0]), "nfs_roi_push")
            return
        a = np.ascontiguousarray(frames, dtype=np.uint16)
        assert a.shape[1:] == (self.H, self.W)
        self._check(self._L.nfs_roi_push(self._h, _ptr(a), a.shape[0]), "nfs_roi_push")

    def push_frames_device(self, frames):
        """frames: CUDA tensor [n, H, W] of 2-byte integers (full frames)."""
        assert tuple(frames.shape[1:]) == (self.H, self.W) and frames.is_contiguous()
        _after_current_stream(self.stream, frames.device)
        self._check(self._L.nfs_roi_push_device(self._h, ctypes.c_void_p(frames.data_ptr()), frames.shape[0]),
                    "nfs_roi_push_device")
        self._inflight.add(frames, self.stream)
