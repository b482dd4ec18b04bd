"""Python binding of libzippir (the GB300 library for the ZipPIR online server phase).

Argument marshalling only: every step of the computation runs in the CUDA kernels
behind the C ABI in ``include/zippir.h``. The binding loads the in-tree
``_lib/libzippir.so`` and raises ``ImportError`` if it has not been built -- there is
no CPU fallback. PyTorch provides device memory and streams; tensors are passed by
their data pointers after dtype/device/shape checks.

Low-level functions carry the C names (``zp_init``, ``zp_setup_db``, ``zp_gen_hint``,
``zp_answer``, ``zp_register_client``, ``zp_compress``, ``zp_respond``,
``zp_respond_host``, ``zp_update_rows`` ...); ``Context``, ``Database`` and
``Client`` wrap them with ownership.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libzippir.so")

ZP_OK, ZP_EINVAL, ZP_ENOMEM, ZP_ECUDA, ZP_ETIMEOUT, ZP_ESTATE, ZP_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
SECRETS = {"uniform": 0, "binary": 1}

# every symbol declared in include/zippir.h
EXPORTS = [
    "zp_version", "zp_last_error", "zp_init", "zp_ctx_destroy", "zp_setup_db", "zp_db_info",
    "zp_db_destroy", "zp_gen_hint", "zp_answer", "zp_register_client", "zp_client_destroy",
    "zp_compress", "zp_respond", "zp_respond_host", "zp_update_rows", "zp_stale_rows",
    "zp_device_status", "zp_kernel_launches", "zp_set_option", "zp_answer_noalloc",
    "zp_compress_products", "zp_compress_finish", "zp_get_option", "zp_client_hint", "zp_combine",
    "zp_db_prepare_rns", "zp_selftest_wait", "zp_autotune", "zp_prg_chacha20", "zp_client_powm",
    "zp_client_expand_ckr", "zp_client_decrypt", "zp_db_prepare_fp16",
    "zp_lc_create", "zp_lc_destroy", "zp_lc_set_key", "zp_lc_unpack_key", "zp_lc_compress",
    "zp_lc_rlwe_extract", "zp_lc_rescale", "zp_db_view",
]


class ZipPIRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("zippir error %d: %s" % (code, msg))
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("key_bits", ctypes.c_uint32),
                ("secret", ctypes.c_uint32), ("p_bits", ctypes.c_uint32), ("scale", ctypes.c_uint32)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libzippir.so (raises ImportError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libzippir.so is not built (%s); run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "zp_version": (i32, []),
        "zp_last_error": (i32, [ctypes.c_char_p, ctypes.c_size_t]),
        "zp_init": (i32, [i32, ctypes.POINTER(_Params), pp]),
        "zp_ctx_destroy": (i32, [vp]),
        "zp_setup_db": (i32, [vp, vp, u32, u32, u64, pp]),
        "zp_db_info": (i32, [vp, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]),
        "zp_db_destroy": (i32, [vp]),
        "zp_db_view": (i32, [vp, pp]),
        "zp_gen_hint": (i32, [vp, vp, vp, vp, u32, vp]),
        "zp_answer": (i32, [vp, vp, u32, vp, vp]),
        "zp_register_client": (i32, [vp, vp, u32, pp]),
        "zp_client_destroy": (i32, [vp]),
        "zp_compress": (i32, [vp, vp, vp, vp, u32, vp, vp]),
        "zp_respond": (i32, [vp, vp, vp, vp, u32, vp, vp, vp]),
        "zp_respond_host": (i32, [vp, vp, vp, vp, u32, vp, vp, vp]),
        "zp_update_rows": (i32, [vp, vp, u32, vp, vp]),
        "zp_stale_rows": (i32, [vp, ctypes.POINTER(u32)]),
        "zp_device_status": (i32, [vp, ctypes.POINTER(u32)]),
        "zp_kernel_launches": (i32, [vp, ctypes.POINTER(u64)]),
        "zp_set_option": (i32, [vp, ctypes.c_char_p, ctypes.c_int64]),
        "zp_answer_noalloc": (i32, [vp, vp, vp, vp]),
        "zp_compress_products": (i32, [vp, vp, u32, vp]),
        "zp_compress_finish": (i32, [vp, vp, vp, u32, vp, vp]),
        "zp_get_option": (i32, [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64)]),
        "zp_client_hint": (i32, [vp, vp, vp, vp, vp, u32, vp]),
        "zp_combine": (i32, [vp, vp, vp, vp, u32, vp, vp]),
        "zp_db_prepare_rns": (i32, [vp, vp]),
        "zp_selftest_wait": (i32, [vp, u64, vp]),
        "zp_autotune": (i32, [vp, vp, ctypes.POINTER(ctypes.c_int64)]),
        "zp_prg_chacha20": (i32, [vp, vp, u32, vp, u64, vp]),
        "zp_client_powm": (i32, [vp, vp, vp, u32, vp, u32, vp]),
        "zp_client_expand_ckr": (i32, [vp, vp, vp, u32, vp, u32, vp]),
        "zp_client_decrypt": (i32, [vp, vp, vp, vp, vp, u32, vp]),
        "zp_db_prepare_fp16": (i32, [vp, vp]),
        "zp_lc_create": (i32, [ctypes.c_int, u32, vp, ctypes.POINTER(vp)]),
        "zp_lc_destroy": (i32, [vp]),
        "zp_lc_set_key": (i32, [vp, vp, u32, u32, vp]),
        "zp_lc_unpack_key": (i32, [vp, vp, u32, u32, vp, u32, vp, vp]),
        "zp_lc_compress": (i32, [vp, vp, vp, u32, u64, u32, vp, u32, ctypes.c_int, vp, vp]),
        "zp_lc_rlwe_extract": (i32, [vp, vp, vp, u32, u64, vp, u32, vp, vp, vp]),
        "zp_lc_rescale": (i32, [vp, vp, u32, u32, u64, u64, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    load_library().zp_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(rc: int):
    if rc != ZP_OK:
        raise ZipPIRError(rc, last_error())


def _ptr(t) -> int | None:
    """Device pointer of a torch tensor / int / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _need(t, dtype_name: str, numel: int | None = None, what: str = "tensor"):
    import torch
    dt = {"u8": torch.uint8, "i32": torch.int32, "i64": torch.int64}[dtype_name]
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % what)
    if t.dtype != dt:
        raise TypeError("%s must have dtype %s (u32 data is passed as int32)" % (what, dt))
    if not t.is_cuda:
        raise TypeError("%s must be on a CUDA device" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if numel is not None and t.numel() < numel:
        raise ValueError("%s has %d elements, needs %d" % (what, t.numel(), numel))


# ----------------------------------------------------------------------------- thin C-named calls
def zp_version() -> int:
    return load_library().zp_version()


SCALES = {"proven": 0, "overlap": 1}


def zp_init(device: int, n: int, key_bits: int = 2048, secret: str = "uniform", p_bits: int = 8,
            scale: str = "proven") -> int:
    P = _Params(n, key_bits, SECRETS[secret], p_bits, SCALES[scale])
    out = ctypes.c_void_p()
    _check(load_library().zp_init(device, ctypes.byref(P), ctypes.byref(out)))
    return out.value


def zp_ctx_destroy(ctx: int):
    _check(load_library().zp_ctx_destroy(ctx))


def zp_setup_db(ctx: int, dD: int, R: int, C: int, ld: int) -> int:
    out = ctypes.c_void_p()
    _check(load_library().zp_setup_db(ctx, dD, R, C, ld, ctypes.byref(out)))
    return out.value


def zp_db_info(db: int) -> tuple[int, int, int]:
    a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(load_library().zp_db_info(db, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def zp_db_destroy(db: int):
    _check(load_library().zp_db_destroy(db))


def zp_db_view(db: int) -> int:
    out = ctypes.c_void_p()
    _check(load_library().zp_db_view(db, ctypes.byref(out)))
    return out.value


def zp_gen_hint(db: int, dA: int, dH: int | None, hRows: np.ndarray | None, stream: int | None):
    if hRows is None:
        _check(load_library().zp_gen_hint(db, dA, dH, None, 0, stream))
    else:
        r = np.ascontiguousarray(hRows, dtype=np.uint32)
        _check(load_library().zp_gen_hint(db, dA, dH, r.ctypes.data, len(r), stream))


def zp_answer(db: int, dQ: int, B: int, dAns: int, stream: int | None):
    _check(load_library().zp_answer(db, dQ, B, dAns, stream))


def zp_answer_noalloc(db: int, dQ: int, dAns: int, stream: int | None):
    """Single-query answer without any device allocation (fixed 1 MiB static scratch,
    C <= 262144); see include/zippir.h."""
    _check(load_library().zp_answer_noalloc(db, dQ, dAns, stream))


def zp_register_client(ctx: int, m: int, L: int) -> int:
    limbs = np.frombuffer(int(m).to_bytes(4 * L, "little"), dtype="<u4").copy()
    out = ctypes.c_void_p()
    _check(load_library().zp_register_client(ctx, limbs.ctypes.data, L, ctypes.byref(out)))
    return out.value


def zp_client_destroy(cl: int):
    _check(load_library().zp_client_destroy(cl))


def _client_array(clients) -> ctypes.Array:
    arr = (ctypes.c_void_p * len(clients))()
    for i, c in enumerate(clients):
        arr[i] = c.handle if isinstance(c, Client) else c
    return arr


def zp_compress(db: int, clients, dAns: int, dCKO: int, B: int, dT: int, stream: int | None):
    _check(load_library().zp_compress(db, ctypes.cast(_client_array(clients), ctypes.c_void_p),
                                      dAns, dCKO, B, dT, stream))


def zp_compress_products(db: int, dCKO: int, B: int, stream: int | None):
    _check(load_library().zp_compress_products(db, dCKO, B, stream))


def zp_compress_finish(db: int, clients, dAns: int, B: int, dT: int, stream: int | None):
    _check(load_library().zp_compress_finish(db, ctypes.cast(_client_array(clients), ctypes.c_void_p),
                                             dAns, B, dT, stream))


def zp_respond(db: int, clients, dQ: int, dCKO: int, B: int, dAns: int, dT: int, stream: int | None):
    _check(load_library().zp_respond(db, ctypes.cast(_client_array(clients), ctypes.c_void_p),
                                     dQ, dCKO, B, dAns, dT, stream))


def zp_respond_host(db: int, clients, hQ: np.ndarray, hCKO: np.ndarray, B: int, hT: np.ndarray,
                    hAns: np.ndarray | None, stream: int | None):
    for a in (hQ, hCKO, hT) + ((hAns,) if hAns is not None else ()):
        if not a.flags["C_CONTIGUOUS"] or a.dtype.itemsize != 4:
            raise ValueError("host buffers must be C-contiguous 32-bit arrays")
    _check(load_library().zp_respond_host(
        db, ctypes.cast(_client_array(clients), ctypes.c_void_p), hQ.ctypes.data, hCKO.ctypes.data,
        B, hT.ctypes.data, None if hAns is None else hAns.ctypes.data, stream))


def zp_client_hint(db: int, client, dCkr: int, dK: int, packed_rows, stream: int | None):
    h = client.handle if isinstance(client, Client) else client
    if packed_rows is None:
        _check(load_library().zp_client_hint(db, h, dCkr, dK, None, 0, stream))
    else:
        r = np.ascontiguousarray(packed_rows, dtype=np.uint32)
        _check(load_library().zp_client_hint(db, h, dCkr, dK, r.ctypes.data, len(r), stream))


def zp_combine(db: int, clients, dK: int, dT: int, B: int, dOut: int, stream: int | None):
    _check(load_library().zp_combine(db, ctypes.cast(_client_array(clients), ctypes.c_void_p),
                                     dK, dT, B, dOut, stream))


def prg_chacha20(key: bytes, nonce: bytes, counter0: int, out, stream=None):
    """Fills the int32 CUDA tensor `out` with ChaCha20 keystream words (zp_prg_chacha20)."""
    if len(key) != 32 or len(nonce) != 12:
        raise ValueError("ChaCha20 takes a 32-byte key and a 12-byte nonce")
    _need(out, "i32", None, "out")
    kb = ctypes.create_string_buffer(bytes(key), 32)
    nb = ctypes.create_string_buffer(bytes(nonce), 12)
    _check(load_library().zp_prg_chacha20(kb, nb, int(counter0), _ptr(out), out.numel(),
                                          _stream(stream)))
    return out


def zp_update_rows(db: int, hRows: np.ndarray, dNew: int, stream: int | None):
    r = np.ascontiguousarray(hRows, dtype=np.uint32)
    _check(load_library().zp_update_rows(db, r.ctypes.data, len(r), dNew, stream))


def zp_stale_rows(db: int) -> int:
    c = ctypes.c_uint32()
    _check(load_library().zp_stale_rows(db, ctypes.byref(c)))
    return c.value


def zp_device_status(ctx: int) -> int:
    c = ctypes.c_uint32()
    _check(load_library().zp_device_status(ctx, ctypes.byref(c)))
    return c.value


def zp_set_option(ctx: int, name: str, value: int):
    _check(load_library().zp_set_option(ctx, name.encode(), int(value)))


def zp_get_option_value(ctx, name: str) -> int:
    """An option of a context (Context or handle), by name."""
    h = ctx.handle if isinstance(ctx, Context) else ctx
    v = ctypes.c_int64()
    _check(load_library().zp_get_option(h, name.encode(), ctypes.byref(v)))
    return v.value


def zp_get_overlap(ctx) -> int:
    """Current "overlap_sms" option of a context (Context or handle)."""
    h = ctx.handle if isinstance(ctx, Context) else ctx
    v = ctypes.c_int64()
    _check(load_library().zp_get_option(h, b"overlap_sms", ctypes.byref(v)))
    return v.value


def zp_kernel_launches(ctx: int) -> int:
    c = ctypes.c_uint64()
    _check(load_library().zp_kernel_launches(ctx, ctypes.byref(c)))
    return c.value


# ----------------------------------------------------------------------------- owning wrappers
class Context:
    """One device and one parameter set (n, key size, secret distribution)."""

    def __init__(self, device: int = 0, n: int = 1024, key_bits: int = 2048, secret: str = "uniform",
                 scale: str = "proven"):
        self.device, self.n, self.key_bits, self.secret, self.scale = device, n, key_bits, secret, scale
        self.handle = zp_init(device, n, key_bits, secret, scale=scale)
        self.L = key_bits // 32

    def register_client(self, m: int) -> "Client":
        return Client(self, m)

    def device_status(self) -> int:
        return zp_device_status(self.handle)

    def selftest_wait(self, cycles: int, stream=None):
        """Runs a bounded wait that nothing satisfies (the failure path of every wait)."""
        _check(load_library().zp_selftest_wait(self.handle, int(cycles), _stream(stream)))

    def kernel_launches(self) -> int:
        return zp_kernel_launches(self.handle)

    def set_option(self, name: str, value):
        """Kernel-variant selection: name in {"answer_path", "compress_path"}, value in
        {"auto", "simt", "tc"} (compress_path also "rns"), or "overlap_sms" / "rns_min_batch" /
        "gemv_max_batch" / "answer_fp16" with an integer."""
        v = {"auto": 0, "simt": 1, "tc": 2, "rns": 3}.get(value, value)
        zp_set_option(self.handle, name, v)

    def close(self):
        if self.handle:
            zp_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Client:
    """A client's public Paillier modulus m, registered on the device."""

    def __init__(self, ctx: Context, m: int):
        self.ctx, self.m = ctx, int(m)
        self.handle = zp_register_client(ctx.handle, self.m, ctx.L)

    def powm(self, bases, exponent: int, out=None, stream=None):
        """bases^exponent mod m^2 for a CUDA int32 tensor of (count, 2L) limbs (zp_client_powm)."""
        import torch
        count = bases.shape[0]
        _need(bases, "i32", count * 2 * self.ctx.L, "bases")
        if out is None:
            out = torch.empty_like(bases)
        ew = max(1, (int(exponent).bit_length() + 31) // 32)
        e = np.array([(int(exponent) >> (32 * i)) & 0xFFFFFFFF for i in range(ew)], dtype=np.uint32)
        _check(load_library().zp_client_powm(self.handle, _ptr(bases), e.ctypes.data, ew, _ptr(out),
                                             count, _stream(stream)))
        return out

    def expand_ckr(self, key: bytes, count: int, nonce: bytes = b"ckr" + bytes(9), counter0: int = 0,
                   out=None, stream=None):
        """ck_r[i] for i < count from a 32-byte seed (zp_client_expand_ckr): (count, 2L) int32."""
        import torch
        if len(key) != 32 or len(nonce) != 12:
            raise ValueError("ChaCha20 takes a 32-byte key and a 12-byte nonce")
        if out is None:
            out = torch.empty((count, 2 * self.ctx.L), dtype=torch.int32,
                              device=torch.device("cuda", self.ctx.device))
        _need(out, "i32", count * 2 * self.ctx.L, "out")
        kb = ctypes.create_string_buffer(bytes(key), 32)
        nb = ctypes.create_string_buffer(bytes(nonce), 12)
        _check(load_library().zp_client_expand_ckr(self.handle, kb, nb, int(counter0), _ptr(out), count,
                                                   _stream(stream)))
        return out

    def decrypt(self, cts, lam: int, mu: int, out=None, stream=None):
        """Paillier decryption of a CUDA int32 tensor of (count, 2L) limbs (zp_client_decrypt):
        (count, L) int32."""
        import torch
        count = cts.shape[0]
        L = self.ctx.L
        _need(cts, "i32", count * 2 * L, "cts")
        if out is None:
            out = torch.empty((count, L), dtype=torch.int32, device=cts.device)
        _need(out, "i32", count * L, "out")
        words = lambda v: np.array([(int(v) >> (32 * i)) & 0xFFFFFFFF for i in range(L)], dtype=np.uint32)
        hl, hm = words(lam), words(mu)
        _check(load_library().zp_client_decrypt(self.handle, hl.ctypes.data, hm.ctypes.data, _ptr(cts),
                                                _ptr(out), count, _stream(stream)))
        return out

    def close(self):
        if self.handle:
            zp_client_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def db_pitch(C: int) -> int:
    """Row pitch (bytes) the library accepts for C columns: C rounded up to 16."""
    return (C + 15) // 16 * 16


class Database:
    """A resident database (R x C bytes, row pitch ``ld``) and its hint.

    ``D`` is a CUDA uint8 tensor of shape (R, ld) (or (R*ld,)); it must outlive the
    Database and must be changed only through ``update_rows``.
    """

    def __init__(self, ctx: Context, D, R: int, C: int, ld: int | None = None, _view_of=None):
        ld = db_pitch(C) if ld is None else ld
        _need(D, "u8", R * ld, "D")
        self.ctx, self.D, self.R, self.C, self.ld = ctx, D, R, C, ld
        self.base = _view_of
        self.handle = zp_db_view(_view_of.handle) if _view_of is not None else \
            zp_setup_db(ctx.handle, _ptr(D), R, C, ld)
        self.ell, self.d1p, self.L = zp_db_info(self.handle)

    def view(self) -> "Database":
        """A second handle on this database with working buffers of its own (zp_db_view), so
        that batches of one database can be in flight at once on different streams. Close
        views before the database."""
        base = self.base if self.base is not None else self
        return Database(self.ctx, base.D, base.R, base.C, base.ld, _view_of=base)

    def gen_hint(self, A, H=None, rows=None, stream=None):
        import torch
        _need(A, "i32", self.C * self.ctx.n, "A")
        if H is not None:
            _need(H, "i32", self.R * self.ctx.n, "H")
        zp_gen_hint(self.handle, _ptr(A), _ptr(H), None if rows is None else np.asarray(rows),
                    _stream(stream))
        return H

    def answer(self, Q, out=None, stream=None):
        import torch
        B = Q.shape[0] if Q.dim() == 2 else 1
        _need(Q, "i32", B * self.C, "Q")
        if out is None:
            out = torch.empty((B, self.R), dtype=torch.int32, device=Q.device)
        _need(out, "i32", B * self.R, "ans")
        zp_answer(self.handle, _ptr(Q), B, _ptr(out), _stream(stream))
        return out

    def compress(self, clients, ans, CKO, out=None, stream=None):
        import torch
        B = len(clients)
        _need(ans, "i32", B * self.R, "ans")
        _need(CKO, "i32", B * self.ctx.n * self.L, "cko")
        if out is None:
            out = torch.empty((B, self.d1p, self.L), dtype=torch.int32, device=ans.device)
        _need(out, "i32", B * self.d1p * self.L, "T")
        zp_compress(self.handle, clients, _ptr(ans), _ptr(CKO), B, _ptr(out), _stream(stream))
        return out

    def respond(self, clients, Q, CKO, ans=None, out=None, stream=None):
        import torch
        B = len(clients)
        _need(Q, "i32", B * self.C, "Q")
        _need(CKO, "i32", B * self.ctx.n * self.L, "cko")
        if ans is None:
            ans = torch.empty((B, self.R), dtype=torch.int32, device=Q.device)
        if out is None:
            out = torch.empty((B, self.d1p, self.L), dtype=torch.int32, device=Q.device)
        zp_respond(self.handle, clients, _ptr(Q), _ptr(CKO), B, _ptr(ans), _ptr(out), _stream(stream))
        return ans, out

    def respond_host(self, clients, hQ: np.ndarray, hCKO: np.ndarray, hT: np.ndarray | None = None,
                     hAns: np.ndarray | None = None, stream=None):
        B = len(clients)
        if hT is None:
            hT = np.empty((B, self.d1p, self.L), dtype=np.uint32)
        zp_respond_host(self.handle, clients, hQ, hCKO, B, hT, hAns, _stream(stream))
        return hT

    def client_hint(self, client, CKR, out=None, packed_rows=None, stream=None):
        """Per-client hint k (d1' x 2L words) from ck_r (n x 2L words)."""
        import torch
        _need(CKR, "i32", self.ctx.n * 2 * self.L, "ckr")
        if out is None:
            out = torch.zeros((self.d1p, 2 * self.L), dtype=torch.int32, device=CKR.device)
        _need(out, "i32", self.d1p * 2 * self.L, "k")
        zp_client_hint(self.handle, client, _ptr(CKR), _ptr(out), packed_rows, _stream(stream))
        return out

    def combine(self, clients, K, T, out=None, stream=None):
        """Combined response k (+) t (B x d1' x 2L words)."""
        import torch
        B = len(clients)
        _need(K, "i32", B * self.d1p * 2 * self.L, "k")
        _need(T, "i32", B * self.d1p * self.L, "T")
        if out is None:
            out = torch.empty((B, self.d1p, 2 * self.L), dtype=torch.int32, device=T.device)
        _need(out, "i32", B * self.d1p * 2 * self.L, "out")
        zp_combine(self.handle, clients, _ptr(K), _ptr(T), B, _ptr(out), _stream(stream))
        return out

    TUNED = ("gemv_max_batch", "rns_min_batch", "overlap_sms", "gemv_cfg_alone", "gemv_cfg_shared",
             "answer_bt_16", "answer_bt_32", "answer_bt_64", "answer_bt_128", "answer_fp16",
             "rns_bt_16", "rns_bt_32", "rns_bt_64", "rns_bt_128", "batch_overlap", "pack_split")

    def autotune(self, stream=None) -> dict:
        """Measures and sets the context's thresholds, tile widths, GEMV configurations and SM
        split (zp_autotune); returns every tuned option."""
        out = (ctypes.c_int64 * 3)()
        _check(load_library().zp_autotune(self.handle, _stream(stream), out))
        return {k: zp_get_option_value(self.ctx, k) for k in self.TUNED}

    def prepare_fp16(self, stream=None):
        """Builds the resident fp16 copy of D (twice its bytes) that batched answers read."""
        _check(load_library().zp_db_prepare_fp16(self.handle, _stream(stream)))

    def prepare_rns(self, stream=None):
        """Builds the RNS residue planes of H' now (else on the first large batch)."""
        _check(load_library().zp_db_prepare_rns(self.handle, _stream(stream)))

    def update_rows(self, rows, new_rows, stream=None):
        _need(new_rows, "u8", len(rows) * self.C, "new_rows")
        zp_update_rows(self.handle, np.asarray(rows), _ptr(new_rows), _stream(stream))

    def stale_rows(self) -> int:
        return zp_stale_rows(self.handle)

    def close(self):
        if self.handle:
            zp_db_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lc_rescale(A, B, q: int, r: int, stream=None):
    """Modulus switching of LWE ciphertexts (zp_lc_rescale): int64 tensors A (count, n) and
    B (count,) modulo q -> new tensors modulo r."""
    import torch
    count = B.shape[0]
    n = A.shape[1] if A.dim() == 2 else 0
    _need(A, "i64", count * n, "A")
    _need(B, "i64", count, "B")
    Ao, Bo = torch.empty_like(A), torch.empty_like(B)
    _check(load_library().zp_lc_rescale(_ptr(A), _ptr(B), count, n, int(q) % (1 << 64), int(r) % (1 << 64),
                                        _ptr(Ao), _ptr(Bo), _stream(stream)))
    return Ao, Bo


def _words(v: int, nw: int | None = None) -> np.ndarray:
    v = int(v)
    if nw is None:
        nw = max(1, (v.bit_length() + 31) // 32)
    return np.array([(v >> (32 * i)) & 0xFFFFFFFF for i in range(nw)], dtype=np.uint32)


class LweCompressor:
    """Standalone compression of LWE ciphertexts / RLWE coefficients into Paillier
    ciphertexts of one modulus m (zp_lc_*). Integers mod q travel as int64 CUDA tensors
    (their u64 bits); Paillier ciphertexts as int32 tensors of 2L limbs."""

    _MODES = {"auto": 0, "horner": 1, "folded": 2}

    def __init__(self, device: int, key_bits: int, m: int):
        self.device, self.key_bits, self.m = device, key_bits, int(m)
        self.L = key_bits // 32
        self.n = 0
        lib = load_library()
        h = ctypes.c_void_p()
        mw = _words(self.m, self.L)
        _check(lib.zp_lc_create(device, key_bits, mw.ctypes.data, ctypes.byref(h)))
        self.handle = h.value

    def set_key(self, ck, T: int, stream=None):
        """Expanded key from ck (n, 2L) for exponents of up to T bits."""
        n = ck.shape[0]
        _need(ck, "i32", n * 2 * self.L, "ck")
        _check(load_library().zp_lc_set_key(self.handle, _ptr(ck), n, int(T), _stream(stream)))
        self.n = n

    def unpack_key(self, pck, n: int, t: int, delta: int, out=None, stream=None):
        import torch
        npk = -(-n // t)
        _need(pck, "i32", npk * 2 * self.L, "pck")
        if out is None:
            out = torch.empty((n, 2 * self.L), dtype=torch.int32, device=pck.device)
        _need(out, "i32", n * 2 * self.L, "out")
        d = _words(delta)
        _check(load_library().zp_lc_unpack_key(self.handle, _ptr(pck), n, t, d.ctypes.data, len(d),
                                               _ptr(out), _stream(stream)))
        return out

    def compress(self, A, B, q: int, ell: int = 1, gamma: int | None = None, mode: str = "auto",
                 out=None, stream=None):
        """A (count, n), B (count,) int64 tensors -> (ceil(count / ell), 2L) int32 tensor."""
        import torch
        count = B.shape[0]
        _need(A, "i64", count * self.n, "A")
        _need(B, "i64", count, "B")
        G = -(-count // ell)
        if out is None:
            out = torch.empty((G, 2 * self.L), dtype=torch.int32, device=B.device)
        _need(out, "i32", G * 2 * self.L, "out")
        g = _words(gamma if gamma is not None else 1)
        _check(load_library().zp_lc_compress(self.handle, _ptr(A), _ptr(B), count, int(q) % (1 << 64),
                                             ell, g.ctypes.data, len(g), self._MODES[mode], _ptr(out),
                                             _stream(stream)))
        return out

    def rlwe_extract(self, A, B, q: int, ks, stream=None):
        """LWE ciphertexts of RLWE coefficients ks: ((len(ks), N), (len(ks),)) int64 tensors."""
        import torch
        N = A.shape[0]
        _need(A, "i64", N, "A")
        _need(B, "i64", N, "B")
        k = np.ascontiguousarray(ks, dtype=np.uint32)
        Ao = torch.empty((len(k), N), dtype=torch.int64, device=A.device)
        Bo = torch.empty((len(k),), dtype=torch.int64, device=A.device)
        _check(load_library().zp_lc_rlwe_extract(self.handle, _ptr(A), _ptr(B), N, int(q) % (1 << 64),
                                                 k.ctypes.data, len(k), _ptr(Ao), _ptr(Bo), _stream(stream)))
        return Ao, Bo

    def close(self):
        if self.handle:
            load_library().zp_lc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
