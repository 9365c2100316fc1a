"""GB300 (sm_103a) construction of MEGAHIT's succinct de Bruijn graph.

A thin binding of the C ABI in ``include/mh.h`` (library ``libmh.so`` next to
this file).  The functions carry the C names and only marshal arguments:
every step runs in the library's CUDA kernels.  PyTorch supplies device
memory (its caching allocator is handed to the library as the allocator
callbacks) and the stream; outputs come back as zero-copy CUDA tensors.

    ctx    = Context(device=0)
    reads  = mh_pack_reads(ctx, ascii, offs)          # uint8 reads, uint64 offsets
    solid  = mh_count_kmers(ctx, reads, k=31, d=2)
    mercy  = mh_mercy_kmers(ctx, reads, solid)
    sdbg   = mh_build_sdbg(ctx, solid, mercy)
    sdbg.W, sdbg.last, sdbg.F, ...                    # CUDA tensors

There is no CPU fallback: without ``libmh.so`` or a CUDA device the calls
raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmh.so")

MH_OK, MH_EINVAL, MH_ENOMEM, MH_EOVERFLOW, MH_ETIMEOUT, MH_EDEVICE, MH_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6

# Every symbol include/mh.h declares.
SYMBOLS = (
    "mh_create", "mh_destroy", "mh_pack_reads", "mh_reads_view_get", "mh_free_reads",
    "mh_count_kmers", "mh_mercy_kmers", "mh_kmers_view_get", "mh_free_kmers", "mh_build_sdbg",
    "mh_sdbg_view_get", "mh_free_sdbg", "mh_strerror", "mh_last_error_message", "mh_stream",
    "mh_memory", "mh_profile_count", "mh_profile_get", "mh_profile_reset", "mh_set_profile",
    "mh_sort_keys_noalloc", "mh_walk_contigs", "mh_contigs_view_get", "mh_free_contigs",
    "mh_pack_reads_contigs", "mh_trim", "mh_run_batch", "mh_sort_shape", "mh_get_count_plan",
    "mh_set_count_plan", "mh_job_bytes", "mh_server_create", "mh_server_submit", "mh_server_wait",
    "mh_server_release", "mh_server_stats", "mh_server_reset_max", "mh_server_context", "mh_server_destroy",
    "mh_sdbg_save", "mh_sdbg_load",
)

MH_BATCH_MERCY, MH_BATCH_BUILD, MH_BATCH_AUTOTUNE = 1, 2, 4
MH_SERVE_AUTO_RELEASE, MH_SERVE_DRY_RUN = 8, 16


class MhError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_strerror(code), code, msg))
        self.code = code


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("hbm_budget", ctypes.c_uint64),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p),
                ("with_mult", ctypes.c_int), ("profile", ctypes.c_int)]


class ReadsView(ctypes.Structure):
    _fields_ = [("n_reads", ctypes.c_uint64), ("n_bases", ctypes.c_uint64), ("n_frags", ctypes.c_uint64),
                ("n_packed", ctypes.c_uint64), ("packed", ctypes.c_void_p), ("frag_offs", ctypes.c_void_p),
                ("frag_read", ctypes.c_void_p)]


class KmersView(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("nw", ctypes.c_int), ("n", ctypes.c_uint64), ("keys", ctypes.c_void_p),
                ("counts", ctypes.c_void_p), ("n_kmers", ctypes.c_uint64), ("n_distinct", ctypes.c_uint64)]


class SdbgView(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("nw", ctypes.c_int), ("m", ctypes.c_uint64), ("t", ctypes.c_uint64),
                ("u", ctypes.c_uint64), ("n_nodes", ctypes.c_uint64), ("F", ctypes.c_uint64 * 6),
                ("W", ctypes.c_void_p), ("last", ctypes.c_void_p), ("valid", ctypes.c_void_p),
                ("dummy", ctypes.c_void_p), ("aux", ctypes.c_void_p), ("mult", ctypes.c_void_p)]


class ReadSet(ctypes.Structure):
    _fields_ = [("ascii", ctypes.c_void_p), ("n_bases", ctypes.c_uint64), ("offs", ctypes.c_void_p),
                ("n_reads", ctypes.c_uint64), ("on_device", ctypes.c_int)]


class SetResult(ctypes.Structure):
    _fields_ = [("solid", ctypes.c_void_p), ("mercy", ctypes.c_void_p), ("sdbg", ctypes.c_void_p),
                ("status", ctypes.c_int)]


class JobInfo(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("end_s", ctypes.c_double),
                ("slot", ctypes.c_int), ("status", ctypes.c_int), ("est_bytes", ctypes.c_uint64)]


class ContigsView(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n", ctypes.c_uint64), ("n_bases", ctypes.c_uint64),
                ("ascii", ctypes.c_void_p), ("offs", ctypes.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmh.so and declare its C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libmh.so is not built (%s); run `python -m paper_1409_7208_gb300._build`" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    PP = ctypes.POINTER(ctypes.c_void_p)
    u64 = ctypes.c_uint64
    lib.mh_create.argtypes = [ctypes.POINTER(Config), PP]
    lib.mh_destroy.argtypes = [P]
    lib.mh_pack_reads.argtypes = [P, P, u64, P, u64, ctypes.c_int, PP]
    lib.mh_reads_view_get.argtypes = [P, ctypes.POINTER(ReadsView)]
    lib.mh_free_reads.argtypes = [P]
    lib.mh_count_kmers.argtypes = [P, P, ctypes.c_int, ctypes.c_int, PP]
    lib.mh_mercy_kmers.argtypes = [P, P, P, PP]
    lib.mh_kmers_view_get.argtypes = [P, ctypes.POINTER(KmersView)]
    lib.mh_free_kmers.argtypes = [P]
    lib.mh_build_sdbg.argtypes = [P, P, P, PP]
    lib.mh_sdbg_view_get.argtypes = [P, ctypes.POINTER(SdbgView)]
    lib.mh_free_sdbg.argtypes = [P]
    lib.mh_strerror.argtypes = [ctypes.c_int]
    lib.mh_strerror.restype = ctypes.c_char_p
    lib.mh_last_error_message.argtypes = [P]
    lib.mh_last_error_message.restype = ctypes.c_char_p
    lib.mh_stream.argtypes = [P]
    lib.mh_stream.restype = P
    lib.mh_memory.argtypes = [P, ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.mh_profile_count.argtypes = [P]
    lib.mh_profile_get.argtypes = [P, ctypes.c_int, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(u64),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64)]
    lib.mh_profile_reset.argtypes = [P]
    lib.mh_set_profile.argtypes = [P, ctypes.c_int]
    lib.mh_sort_keys_noalloc.argtypes = [P, P, u64, ctypes.c_int, ctypes.c_int, P]
    lib.mh_walk_contigs.argtypes = [P, P, P, u64, u64, u64, PP]
    lib.mh_contigs_view_get.argtypes = [P, ctypes.POINTER(ContigsView)]
    lib.mh_free_contigs.argtypes = [P]
    lib.mh_pack_reads_contigs.argtypes = [P, P, u64, P, u64, P, ctypes.c_int, PP]
    lib.mh_trim.argtypes = [P]
    lib.mh_run_batch.argtypes = [P, ctypes.POINTER(ReadSet), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.POINTER(SetResult)]
    lib.mh_sort_shape.argtypes = [P]
    lib.mh_get_count_plan.argtypes = [P, ctypes.POINTER(CountPlan)]
    lib.mh_set_count_plan.argtypes = [P, ctypes.POINTER(CountPlan)]
    lib.mh_job_bytes.argtypes = [ctypes.POINTER(ReadSet), ctypes.c_int]
    lib.mh_job_bytes.restype = u64
    lib.mh_server_create.argtypes = [P, ctypes.c_int, u64, ctypes.c_int, PP]
    lib.mh_server_submit.argtypes = [P, ctypes.POINTER(ReadSet), ctypes.c_int, ctypes.c_int, ctypes.POINTER(u64)]
    lib.mh_server_wait.argtypes = [P, u64, ctypes.c_double, ctypes.POINTER(SetResult), ctypes.POINTER(JobInfo)]
    lib.mh_server_release.argtypes = [P, u64]
    lib.mh_server_stats.argtypes = [P, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64),
                                    ctypes.POINTER(u64)]
    lib.mh_server_reset_max.argtypes = [P]
    lib.mh_server_context.argtypes = [P, ctypes.c_int]
    lib.mh_server_context.restype = P
    lib.mh_server_destroy.argtypes = [P]
    lib.mh_sdbg_save.argtypes = [P, ctypes.c_char_p]
    lib.mh_sdbg_load.argtypes = [P, ctypes.c_char_p, PP]
    _lib = lib
    return lib


def _strerror(code: int) -> str:
    try:
        return load_library().mh_strerror(code).decode()
    except ImportError:
        return "error"


# ------------------------------------------------------------- tensors

class _DeviceArray:
    """Borrowed device memory exposed through __cuda_array_interface__; keeps
    its owner (the handle) alive while a tensor refers to it."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}
        self._owner = owner


def _tensor(ptr, shape, typestr, owner, device):
    import torch
    dt = {"<i8": torch.int64, "<i4": torch.int32, "|u1": torch.uint8}[typestr]
    if ptr is None or int(np.prod(shape)) == 0:
        return torch.empty(tuple(shape), dtype=dt, device=device)
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr, owner), device=device)


# ------------------------------------------------------------- context

class Context:
    """A library context on one CUDA device and stream.

    ``stream``: a ``torch.cuda.Stream`` (default: the current stream).
    ``torch_allocator``: allocate through PyTorch's caching allocator
    (default); otherwise the library's own stream-ordered pool.
    ``hbm_budget``: bytes the context may hold at once (0 = unlimited).
    """

    def __init__(self, device: int = 0, stream=None, hbm_budget: int = 0, torch_allocator: bool = True,
                 with_mult: bool = False, profile: bool = False):
        import torch
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("the SdBG library needs a CUDA device; none is available")
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.torch_stream = stream
        cfg = Config()
        cfg.device = device
        cfg.stream = stream.cuda_stream
        cfg.hbm_budget = hbm_budget
        cfg.with_mult = 1 if with_mult else 0
        cfg.profile = 1 if profile else 0
        if torch_allocator:
            dev = device

            def _alloc(nbytes, strm, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(strm or 0))
                except Exception:
                    return None

            def _free(ptr, nbytes, strm, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            cfg.alloc, cfg.free = self._cb
        h = ctypes.c_void_p()
        rc = lib.mh_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != MH_OK:
            raise MhError(rc, "mh_create failed")
        self._h = h
        self._lib = lib

    def _check(self, rc: int):
        if rc != MH_OK:
            raise MhError(rc, self._lib.mh_last_error_message(self._h).decode())

    @property
    def handle(self):
        return self._h

    def stream(self):
        """The library's stream as a torch stream (record timing events on it)."""
        import torch
        ptr = self._lib.mh_stream(self._h)
        if ptr == self.torch_stream.cuda_stream:
            return self.torch_stream
        return torch.cuda.ExternalStream(ptr, device=self.device)

    def trim(self):
        """Give the memory the library's own pool keeps cached back to the driver."""
        self._check(self._lib.mh_trim(self._h))

    def memory(self):
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        self._lib.mh_memory(self._h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def set_profile(self, on: bool):
        self._lib.mh_set_profile(self._h, 1 if on else 0)

    def profile(self) -> dict:
        """{kernel name: (launches, total ms, algorithmic bytes)} gathered
        while profiling is on."""
        n = self._lib.mh_profile_count(self._h)
        out = {}
        buf = ctypes.create_string_buffer(128)
        for i in range(n):
            la, ms, by = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_uint64()
            self._check(self._lib.mh_profile_get(self._h, i, buf, 128, ctypes.byref(la), ctypes.byref(ms),
                                                 ctypes.byref(by)))
            out[buf.value.decode()] = (la.value, ms.value, by.value)
        return out

    def profile_reset(self):
        self._lib.mh_profile_reset(self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Handle:
    _free_name = ""

    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self._h = h

    def free(self):
        # a borrowed handle (a server's result) is freed by its owner
        if getattr(self, "_h", None) and self.ctx._h and not getattr(self, "borrowed", False):
            getattr(self.ctx._lib, self._free_name)(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Reads(_Handle):
    _free_name = "mh_free_reads"

    def view(self) -> ReadsView:
        v = ReadsView()
        self.ctx._check(self.ctx._lib.mh_reads_view_get(self._h, ctypes.byref(v)))
        return v

    @property
    def n_frags(self):
        return self.view().n_frags

    def tensors(self) -> dict:
        v = self.view()
        d = self.ctx.device
        return {"packed": _tensor(v.packed, ((v.n_packed + 15) // 16,), "<i4", self, d),
                "frag_offs": _tensor(v.frag_offs, (v.n_frags + 1,), "<i8", self, d),
                "frag_read": _tensor(v.frag_read, (v.n_frags,), "<i4", self, d),
                "n_packed": v.n_packed, "n_frags": v.n_frags}


class Kmers(_Handle):
    _free_name = "mh_free_kmers"

    def view(self) -> KmersView:
        v = KmersView()
        self.ctx._check(self.ctx._lib.mh_kmers_view_get(self._h, ctypes.byref(v)))
        return v

    @property
    def n(self):
        return self.view().n

    @property
    def keys(self):
        """(n, nw) int64 CUDA tensor with the bits of the uint64 key words."""
        v = self.view()
        return _tensor(v.keys, (v.n, v.nw), "<i8", self, self.ctx.device)

    @property
    def counts(self):
        """(n,) int32 CUDA tensor with the bits of the uint32 counts."""
        v = self.view()
        return _tensor(v.counts, (v.n,), "<i4", self, self.ctx.device)

    def numpy(self) -> dict:
        v = self.view()
        return {"k": v.k, "nw": v.nw, "keys": self.keys.cpu().numpy().view(np.uint64),
                "counts": self.counts.cpu().numpy().view(np.uint32), "n_kmers": v.n_kmers,
                "n_distinct": v.n_distinct}


class Sdbg(_Handle):
    _free_name = "mh_free_sdbg"

    def view(self) -> SdbgView:
        v = SdbgView()
        self.ctx._check(self.ctx._lib.mh_sdbg_view_get(self._h, ctypes.byref(v)))
        return v

    def tensors(self) -> dict:
        v = self.view()
        d = self.ctx.device
        nwords = (v.m + 31) // 32
        out = {"k": v.k, "nw": v.nw, "m": v.m, "t": v.t, "u": v.u, "n_nodes": v.n_nodes, "F": list(v.F),
               "W": _tensor(v.W, (v.m,), "|u1", self, d),
               "last": _tensor(v.last, (nwords,), "<i4", self, d),
               "valid": _tensor(v.valid, (nwords,), "<i4", self, d),
               "dummy": _tensor(v.dummy, (nwords,), "<i4", self, d),
               "aux": _tensor(v.aux, (v.t, v.nw), "<i8", self, d)}
        out["mult"] = _tensor(v.mult, (v.m,), "<i4", self, d) if v.mult else None
        return out

    def numpy(self) -> dict:
        """Host copy with bit-vectors unpacked to one byte per entry."""
        t = self.tensors()
        m = t["m"]

        def bits(x):
            w = x.cpu().numpy().view(np.uint32)
            b = np.unpackbits(w.view(np.uint8), bitorder="little")
            return b[:m].astype(np.uint8)

        out = {"k": t["k"], "nw": t["nw"], "m": m, "t": t["t"], "u": t["u"], "n_nodes": t["n_nodes"],
               "F": np.array(t["F"], dtype=np.uint64), "W": t["W"].cpu().numpy(),
               "last": bits(t["last"]), "valid": bits(t["valid"]), "dummy": bits(t["dummy"]),
               "aux": t["aux"].cpu().numpy().view(np.uint64).reshape(t["t"], t["nw"])}
        if t["mult"] is not None:
            out["mult"] = t["mult"].cpu().numpy().view(np.uint32)
        return out


class Contigs(_Handle):
    _free_name = "mh_free_contigs"

    def view(self) -> ContigsView:
        v = ContigsView()
        self.ctx._check(self.ctx._lib.mh_contigs_view_get(self._h, ctypes.byref(v)))
        return v

    def tensors(self) -> dict:
        v = self.view()
        d = self.ctx.device
        return {"k": v.k, "n": v.n, "n_bases": v.n_bases,
                "ascii": _tensor(v.ascii, (v.n_bases,), "|u1", self, d),
                "offs": _tensor(v.offs, (v.n + 1,), "<i8", self, d)}

    def numpy(self) -> dict:
        t = self.tensors()
        return {"k": t["k"], "ascii": t["ascii"].cpu().numpy(), "offs": t["offs"].cpu().numpy().view(np.uint64)}

    def strings(self) -> list:
        c = self.numpy()
        a, o = c["ascii"].tobytes(), c["offs"]
        return [a[int(o[i]):int(o[i + 1])].decode() for i in range(len(o) - 1)]


# ------------------------------------------------------- the C entry points

def _ptr_of(x):
    """(pointer, on_device) of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data, 0
    import torch
    if isinstance(x, torch.Tensor):
        return x.data_ptr(), 1 if x.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def mh_pack_reads(ctx: Context, ascii, offs) -> Reads:
    """2-bit packing of reads (``ascii``: uint8, all reads back to back;
    ``offs``: uint64 offsets, n_reads + 1).  Both on the host (numpy or CPU
    tensor; pinned memory makes the copy asynchronous) or both on the device."""
    if isinstance(ascii, np.ndarray):
        ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
        offs = np.ascontiguousarray(offs, dtype=np.uint64)
    pa, da = _ptr_of(ascii)
    po, do = _ptr_of(offs)
    if da != do:
        raise ValueError("ascii and offs must both be on the host or both on the device")
    n_bases = int(ascii.shape[0])
    n_reads = int(offs.shape[0]) - 1
    h = ctypes.c_void_p()
    ctx._check(ctx._lib.mh_pack_reads(ctx._h, pa if n_bases else None, n_bases, po, n_reads, da, ctypes.byref(h)))
    return Reads(ctx, h)


def mh_count_kmers(ctx: Context, reads: Reads, k: int, d: int = 2) -> Kmers:
    """Solid (k+1)-mers: all (k+1)-mers on both strands, count >= d."""
    h = ctypes.c_void_p()
    ctx._check(ctx._lib.mh_count_kmers(ctx._h, reads._h, int(k), int(d), ctypes.byref(h)))
    return Kmers(ctx, h)


def mh_mercy_kmers(ctx: Context, reads: Reads, solid: Kmers) -> Kmers:
    """Mercy (k+1)-mers recovered between dead ends of the solid graph."""
    h = ctypes.c_void_p()
    ctx._check(ctx._lib.mh_mercy_kmers(ctx._h, reads._h, solid._h, ctypes.byref(h)))
    return Kmers(ctx, h)


def mh_build_sdbg(ctx: Context, solid: Kmers, mercy: Kmers | None = None) -> Sdbg:
    """BOSS arrays of the edge set solid + mercy in colex order."""
    h = ctypes.c_void_p()
    ctx._check(ctx._lib.mh_build_sdbg(ctx._h, solid._h, mercy._h if mercy is not None else None,
                                      ctypes.byref(h)))
    return Sdbg(ctx, h)



def mh_sdbg_save(g: Sdbg, path: str):
    """Write the graph to one flat file (see include/mh.h)."""
    g.ctx._check(g.ctx._lib.mh_sdbg_save(g._h, os.fsencode(path)))


def mh_sdbg_load(ctx: Context, path: str) -> Sdbg:
    """Read a graph written by :func:`mh_sdbg_save` onto ctx's device."""
    h = ctypes.c_void_p()
    ctx._check(ctx._lib.mh_sdbg_load(ctx._h, os.fsencode(path), ctypes.byref(h)))
    return Sdbg(ctx, h)


def mh_walk_contigs(ctx: Context, solid: Kmers, mercy: Kmers | None, n_walks: int, max_len: int,
                    seed: int) -> Contigs:
    """Contigs as seeded random walks of the graph solid + mercy."""
    h = ctypes.c_void_p()
    ctx._check(ctx._lib.mh_walk_contigs(ctx._h, solid._h, mercy._h if mercy is not None else None, int(n_walks),
                                        int(max_len), int(seed), ctypes.byref(h)))
    return Contigs(ctx, h)


def mh_run_batch(ctx: Context, sets, k: int, d: int = 2, workers: int = 4, mercy: bool = True,
                 build: bool = True, autotune: bool = False) -> list:
    """The whole path on many independent read sets at once (``sets``: a list
    of (ascii, offs) pairs, each as for :func:`mh_pack_reads`), on
    ``workers`` concurrent worker streams, largest set first.  Returns one
    dict per set, in input order: ``solid``, ``mercy``, ``sdbg`` handles
    (None where skipped).  Raises :class:`MhError` if a set failed (after
    freeing every output)."""
    arr = (ReadSet * max(1, len(sets)))()
    keep = []
    for i, (ascii, offs) in enumerate(sets):
        if isinstance(ascii, np.ndarray):
            ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
            offs = np.ascontiguousarray(offs, dtype=np.uint64)
        keep.append((ascii, offs))
        pa, da = _ptr_of(ascii)
        po, do = _ptr_of(offs)
        if da != do:
            raise ValueError("set %d: ascii and offs must both be on the host or both on the device" % i)
        n_bases = int(ascii.shape[0])
        arr[i] = ReadSet(pa if n_bases else None, n_bases, po, int(offs.shape[0]) - 1, da)
    res = (SetResult * max(1, len(sets)))()
    flags = (MH_BATCH_MERCY if mercy else 0) | (MH_BATCH_BUILD if build else 0) | \
        (MH_BATCH_AUTOTUNE if autotune else 0)
    rc = ctx._lib.mh_run_batch(ctx._h, arr, len(sets), int(k), int(d), int(workers), flags, res)
    out = []
    for i in range(len(sets)):
        r = res[i]
        out.append({"solid": Kmers(ctx, r.solid) if r.solid else None,
                    "mercy": Kmers(ctx, r.mercy) if r.mercy else None,
                    "sdbg": Sdbg(ctx, r.sdbg) if r.sdbg else None, "status": r.status})
    if rc != MH_OK:
        for o in out:
            for key in ("sdbg", "mercy", "solid"):
                if o[key] is not None:
                    o[key].free()
        ctx._check(rc)
    return out


PLAN_FIELDS = ("path", "sort_shape", "unit_bits_delta", "spread_bits_delta", "bucket_bits")


class CountPlan(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int) for f in PLAN_FIELDS]


def mh_get_count_plan(ctx: Context) -> dict:
    """The context's counting plan (mh_count_plan) as a dict."""
    p = CountPlan()
    ctx._check(ctx._lib.mh_get_count_plan(ctx._h, ctypes.byref(p)))
    return {f: getattr(p, f) for f in PLAN_FIELDS}


def mh_set_count_plan(ctx: Context, **fields) -> None:
    """Set the context's counting plan; fields not given keep their value."""
    cur = mh_get_count_plan(ctx)
    cur.update(fields)
    p = CountPlan(*[int(cur[f]) for f in PLAN_FIELDS])
    ctx._check(ctx._lib.mh_set_count_plan(ctx._h, ctypes.byref(p)))


def mh_sort_shape(ctx: Context) -> int:
    """The scatter tile shape the context uses for 1-word keys (-1: default)."""
    return int(ctx._lib.mh_sort_shape(ctx._h))


def mh_pack_reads_contigs(ctx: Context, ascii, offs, contigs: Contigs | None, copies: int) -> Reads:
    """mh_pack_reads of device reads plus ``copies`` copies of every contig."""
    pa, da = _ptr_of(ascii)
    po, do = _ptr_of(offs)
    if not (da and do):
        raise ValueError("ascii and offs must be device tensors")
    n_bases = int(ascii.shape[0])
    n_reads = int(offs.shape[0]) - 1
    h = ctypes.c_void_p()
    ctx._check(ctx._lib.mh_pack_reads_contigs(ctx._h, pa if n_bases else None, n_bases, po, n_reads,
                                              contigs._h if contigs is not None else None, int(copies),
                                              ctypes.byref(h)))
    return Reads(ctx, h)


def mh_sort_keys_noalloc(keys_in, keys_out, nw: int, key_bits: int, stream=None) -> None:
    """Sort device keys without any device allocation (the C entry point of
    the same name): for callers that must not allocate, e.g. inside an engine
    that owns all device memory.  ``keys_in``/``keys_out``: CUDA tensors of
    n * nw int64 (uint64 bits), distinct; n * nw <= 2^21.  The first call per
    device looks up the library's static scratch array; overlapping calls
    race on that array."""
    import torch
    lib = load_library()
    if int(nw) not in (1, 2, 4):
        raise ValueError("nw must be 1, 2 or 4")
    for name, t in (("keys_in", keys_in), ("keys_out", keys_out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
        if t.dtype != torch.int64:
            raise ValueError("%s must be int64 (uint64 bits)" % name)
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if keys_in.device != keys_out.device or keys_in.device.index != torch.cuda.current_device():
        raise ValueError("keys_in and keys_out must be on the current CUDA device")
    if keys_in.numel() % int(nw):
        raise ValueError("keys_in holds %d words, not a multiple of nw = %d" % (keys_in.numel(), nw))
    if keys_out.numel() < keys_in.numel():
        raise ValueError("keys_out holds fewer words than keys_in")
    if stream is None:
        stream = torch.cuda.current_stream()
    n = keys_in.numel() // int(nw)
    rc = lib.mh_sort_keys_noalloc(keys_in.data_ptr(), keys_out.data_ptr(), n, int(nw), int(key_bits),
                                  stream.cuda_stream)
    if rc != MH_OK:
        raise MhError(rc, "mh_sort_keys_noalloc")
