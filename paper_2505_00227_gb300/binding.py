"""Thin ctypes binding of the C ABI in ``include/hpmdr.h``.

Only argument marshalling happens here: every step of refactoring and
retrieval runs in the sm_103a kernels of ``libhpmdr.so``.  PyTorch supplies
device memory (tensors) and the CUDA stream.  If the shared library has not
been built, importing the binding raises; there is no fallback.
"""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhpmdr.so")

OK, ERR_ARG, ERR_NOMEM, ERR_CUDA, ERR_CORRUPT, ERR_UNATTAINABLE, ERR_TIMEOUT, ERR_BUSY = (
    0, -1, -2, -3, -4, -5, -6, -7)
ERR_CANCELLED = -8
F32, F64 = 0, 1
DC, HUFFMAN, RLE, PLACEHOLDER = 0, 1, 2, 3


class Config(C.Structure):
    _fields_ = [("group_m", C.c_int), ("size_threshold", C.c_uint64), ("cr_num", C.c_uint32),
                ("cr_den", C.c_uint32), ("method", C.c_int32), ("reserved0", C.c_int32),
                ("reserved", C.c_uint64 * 3)]


class Allocator(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)),
                ("user", C.c_void_p)]


class RetrieveInfo(C.Structure):
    _fields_ = [("est_linf", C.c_double), ("requested_abs", C.c_double),
                ("est_units_hi", C.c_uint64), ("est_units_lo", C.c_uint64),
                ("bytes_fetched_total", C.c_uint64), ("bytes_fetched_new", C.c_uint64),
                ("groups_per_level", C.c_int * 64), ("nlevels", C.c_int), ("status", C.c_int)]

    @property
    def groups(self):
        return list(self.groups_per_level[: self.nlevels])

    @property
    def est_units(self):
        return (self.est_units_hi << 64) | self.est_units_lo


class QoiReport(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("tau_abs", C.c_double),
                ("est", C.c_double), ("eps", C.c_double * 3), ("prefix", C.c_int * 3),
                ("pad", C.c_int), ("bytes_fetched_total", C.c_uint64)]


EST_CP, EST_MA, EST_MAPE = 0, 1, 2


class Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("h", C.c_void_p * 3), ("rel_bound", C.c_double),
                ("out", C.c_void_p * 3), ("out_vmag", C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [("max_slots", C.c_int), ("keep_cache", C.c_int), ("hbm_budget", C.c_uint64),
                ("queue_timeout_s", C.c_double)]


REQ_FIELD, REQ_VMAG = 0, 1


class HpmdrError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.hpmdr_strerror(status).decode() if _lib else str(status)
        detail = _lib.hpmdr_last_error().decode() if _lib else ""
        super().__init__(f"{where}: {msg} ({status}) {detail}".strip())


_lib = None
vp = C.c_void_p
u64p = C.POINTER(C.c_uint64)
ip = C.POINTER(C.c_int)

_SIGS = {
    "hpmdr_ctx_create": (C.c_int, [C.POINTER(vp), C.POINTER(Config), C.POINTER(Allocator), vp]),
    "hpmdr_ctx_destroy": (None, [vp]),
    "hpmdr_ctx_set_stream": (C.c_int, [vp, vp]),
    "hpmdr_refactor": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_uint64 * 3, C.c_int, C.POINTER(vp)]),
    "hpmdr_retrieve": (C.c_int, [vp, vp, C.c_double, vp, C.c_int, C.POINTER(RetrieveInfo)]),
    "hpmdr_retrieve_abs": (C.c_int, [vp, vp, C.c_double, vp, C.c_int, C.POINTER(RetrieveInfo)]),
    "hpmdr_qoi_prepare_vmag": (C.c_int, [vp, vp * 3, vp, vp, vp, C.c_int]),
    "hpmdr_retrieve_qoi_vmag": (C.c_int, [vp, vp * 3, C.c_double, vp * 3, vp, C.c_int,
                                          RetrieveInfo * 4]),
    "hpmdr_qoi_prepare_vtotal": (C.c_int, [vp, vp * 3, vp, vp, vp, C.c_int]),
    "hpmdr_retrieve_qoi_vtotal": (C.c_int, [vp, vp * 3, C.c_double, C.c_int, C.c_double, vp * 3,
                                            vp, C.c_int, C.POINTER(QoiReport)]),
    "hpmdr_handle_field_info": (C.c_int, [vp, ip, C.c_uint64 * 3, ip, ip, ip, C.c_double * 4]),
    "hpmdr_handle_level_info": (C.c_int, [vp, C.c_int, u64p, ip, ip, ip]),
    "hpmdr_handle_group": (C.c_int, [vp, C.c_int, C.c_int, vp, u64p, ip, C.c_uint64 * 2]),
    "hpmdr_handle_planes": (C.c_int, [vp, C.c_int, vp, u64p]),
    "hpmdr_handle_sequence": (C.c_int, [vp, ip, C.c_int, ip]),
    "hpmdr_handle_export": (C.c_int, [vp, vp, u64p]),
    "hpmdr_handle_import": (C.c_int, [vp, vp, C.c_uint64, C.POINTER(vp)]),
    "hpmdr_handle_reset": (C.c_int, [vp, vp, C.c_int]),
    "hpmdr_handle_free": (None, [vp]),
    "hpmdr_handle_compact": (C.c_int, [vp, vp]),
    "hpmdr_handle_drop_cache": (C.c_int, [vp, vp]),
    "hpmdr_handle_memory": (C.c_int, [vp, u64p, u64p, u64p]),
    "hpmdr_retrieve_async": (C.c_int, [vp, vp, C.c_double, vp, vp]),
    "hpmdr_retrieve_async_host": (C.c_int, [vp, vp, C.c_double, vp, vp]),
    "hpmdr_ctx_wait": (C.c_int, [vp]),
    "hpmdr_refactor_pipeline": (C.c_int, [vp, C.c_int, vp, C.c_int, u64p, u64p, C.c_int, C.c_int,
                                          vp, u64p, u64p, u64p]),
    "hpmdr_retrieve_pipeline": (C.c_int, [vp, C.c_int, vp, u64p, u64p, C.c_int, u64p, u64p,
                                          C.POINTER(C.c_double), C.c_int, vp, vp]),
    "hpmdr_ctx_profile_stages": (C.c_int, [vp, C.c_uint64]),
    "hpmdr_fixed_to_float": (C.c_int, [vp, vp, C.c_uint64, C.c_int, C.c_int, vp]),
    "hpmdr_qoi_vtotal_bound": (C.c_int, [vp, vp, vp, vp, C.c_uint64, C.c_double * 3, vp,
                                         C.POINTER(C.c_double), u64p]),
    "hpmdr_refactor_chunked": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_uint64 * 3, C.c_uint64 * 3,
                                         C.c_int, C.c_int, C.POINTER(vp), C.c_uint64, u64p]),
    "hpmdr_retrieve_chunked": (C.c_int, [vp, C.POINTER(vp), C.c_uint64, C.c_int, C.c_uint64 * 3,
                                         C.c_uint64 * 3, C.c_double, vp, C.c_int, C.c_int,
                                         C.POINTER(RetrieveInfo)]),
    "hpmdr_server_create": (C.c_int, [vp, C.POINTER(ServerConfig), C.POINTER(vp)]),
    "hpmdr_server_destroy": (None, [vp]),
    "hpmdr_server_add_field": (C.c_int, [vp, vp, vp]),
    "hpmdr_server_submit": (C.c_int, [vp, C.POINTER(Request), u64p]),
    "hpmdr_server_poll": (C.c_int, [vp, C.c_uint64, C.c_int, RetrieveInfo * 4, C.c_double * 3]),
    "hpmdr_server_stats": (C.c_int, [vp, C.c_uint64 * 6]),
    "hpmdr_server_cancel": (C.c_int, [vp, C.c_uint64]),
    "hpmdr_batch_create": (C.c_int, [vp, C.c_uint64, u64p, C.c_int, C.POINTER(vp)]),
    "hpmdr_batch_destroy": (None, [vp]),
    "hpmdr_batch_handle": (C.c_int, [vp, C.c_uint64, C.POINTER(vp)]),
    "hpmdr_batch_refactor": (C.c_int, [vp, C.POINTER(vp)]),
    "hpmdr_batch_retrieve": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(vp),
                                       C.POINTER(RetrieveInfo)]),
    "hpmdr_batch_autotune": (C.c_int, [vp, C.POINTER(vp), C.POINTER(C.c_double), C.POINTER(vp),
                                       C.c_uint32 * 3]),
    "hpmdr_batch_set_tuning": (C.c_int, [vp, C.c_uint32 * 3]),
    "hpmdr_batch_get_tuning": (C.c_int, [vp, C.c_uint32 * 3]),
    "hpmdr_batch_last_ms": (C.c_int, [vp, C.c_double * 2]),
    "hpmdr_bitplane_encode": (C.c_int, [vp, vp, C.c_uint64, C.c_int, vp, vp]),
    "hpmdr_bitplane_decode": (C.c_int, [vp, C.c_uint64, C.c_int, C.c_int, vp, vp, vp]),
    "hpmdr_bitplane_encode_design": (C.c_int, [vp, vp, C.c_uint64, C.c_int, vp, vp]),
    "hpmdr_bitplane_decode_design": (C.c_int, [vp, C.c_uint64, C.c_int, C.c_int, vp, vp, vp]),
    "hpmdr_encode_group": (C.c_int, [vp, vp, C.c_uint64, C.c_int, vp, C.c_uint64, u64p, ip]),
    "hpmdr_decode_group": (C.c_int, [vp, vp, C.c_uint64, C.c_int, vp, C.c_uint64]),
    "hpmdr_encode_group_noalloc": (C.c_int, [vp, C.c_uint64, C.c_int, C.c_uint64, C.c_uint32,
                                             C.c_uint32, vp, C.c_uint64, u64p, ip, vp]),
    "hpmdr_kernel_launches": (C.c_uint64, []),
    "hpmdr_ctx_profile": (C.c_int, [vp, C.c_int]),
    "hpmdr_ctx_profile_entry": (C.c_int, [vp, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_double),
                                          u64p, C.POINTER(C.c_double)]),
    "hpmdr_strerror": (C.c_char_p, [C.c_int]),
    "hpmdr_last_error": (C.c_char_p, []),
}


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2505_00227_gb300.build")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def kernel_launches():
    """Kernels launched by libhpmdr.so in this process so far."""
    return int(lib().hpmdr_kernel_launches())


def _check(status, where, allow=()):
    if status != OK and status not in allow:
        raise HpmdrError(status, where)
    return status


def _dims3(shape):
    s = tuple(int(x) for x in shape)
    if not 1 <= len(s) <= 3:
        raise ValueError("1 to 3 dimensions")
    full = (1,) * (3 - len(s)) + s
    return len(s), (C.c_uint64 * 3)(*full)


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return vp(int(getattr(stream, "cuda_stream", stream)))


def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"unsupported dtype {t.dtype}")


# ------------------------------------------------------------------ objects
class Context:
    """hpmdr_ctx bound to a CUDA stream (torch's current stream by default)."""

    def __init__(self, size_threshold=0, cr_num=0, cr_den=0, stream=None, method=None):
        """method: None for Algorithm 2, else DC / HUFFMAN / RLE for every group."""
        cfg = Config(4, size_threshold, cr_num, cr_den, 0 if method is None else method + 1)
        self._p = vp()
        self._keep = []  # infos and outputs of pending asynchronous retrievals
        _check(lib().hpmdr_ctx_create(C.byref(self._p), C.byref(cfg), None, _stream_ptr(stream)),
               "hpmdr_ctx_create")

    def refactor_pipeline(self, fields, chunk, queues=3):
        """Out-of-core refactoring of host tensors of one shape (Sec. 5.3):
        returns (streams as a page-locked uint8 tensor, offsets, sizes)."""
        import torch
        nv = len(fields)
        shape = tuple(fields[0].shape)
        dt = F32 if fields[0].dtype == torch.float32 else F64
        nd = len(shape)
        dims = (C.c_uint64 * 3)(*([1] * (3 - nd) + list(shape)))
        ch = (C.c_uint64 * 3)(*([1] * (3 - nd) + list(chunk)))
        ptrs = (vp * nv)(*[vp(f.data_ptr()) for f in fields])
        total = C.c_uint64(0)
        _check(lib().hpmdr_refactor_pipeline(self._p, nv, ptrs, nd, dims, ch, dt, queues, None,
                                             C.byref(total), None, None), "hpmdr_refactor_pipeline")
        out = torch.empty(total.value, dtype=torch.uint8).pin_memory()
        ncell = 1
        for d, c in zip(shape, chunk):
            ncell *= (d + c - 1) // c
        offs = (C.c_uint64 * (nv * ncell))()
        sizes = (C.c_uint64 * (nv * ncell))()
        _check(lib().hpmdr_refactor_pipeline(self._p, nv, ptrs, nd, dims, ch, dt, queues,
                                             vp(out.data_ptr()), C.byref(total), offs, sizes),
               "hpmdr_refactor_pipeline")
        return out[: total.value], list(offs), list(sizes)

    def retrieve_pipeline(self, streams, offsets, sizes, shape, chunk, bounds, outs, queues=3):
        """Retrieve every unit of the streams into the host tensors `outs` (one
        per variable) at the relative bounds; returns (infos, status)."""
        nv = len(outs)
        nd = len(shape)
        dims = (C.c_uint64 * 3)(*([1] * (3 - nd) + list(shape)))
        ch = (C.c_uint64 * 3)(*([1] * (3 - nd) + list(chunk)))
        n = len(offsets)
        offs = (C.c_uint64 * n)(*offsets)
        szs = (C.c_uint64 * n)(*sizes)
        b = (C.c_double * nv)(*[float(x) for x in bounds])
        ptrs = (vp * nv)(*[vp(o.data_ptr()) for o in outs])
        infos = (RetrieveInfo * n)()
        st = lib().hpmdr_retrieve_pipeline(self._p, nv, vp(streams.data_ptr()), offs, szs, nd, dims,
                                           ch, b, queues, ptrs, infos)
        _check(st, "hpmdr_retrieve_pipeline", allow=(ERR_UNATTAINABLE,))
        return list(infos), st

    def wait(self):
        """Wait for the context stream; fills the infos of the asynchronous
        retrievals.  Returns HPMDR_OK or the first pending status that was not
        OK (HPMDR_ERR_UNATTAINABLE included); raises on other errors."""
        st = lib().hpmdr_ctx_wait(self._p)
        self._keep = []
        _check(st, "hpmdr_ctx_wait", allow=(ERR_UNATTAINABLE,))
        return st

    def profile(self, enable=True, stages=None):
        """Record per-stage CUDA events on this context's stream (clears totals);
        stages: names of the only stages that record (None: all)."""
        if stages is None:
            _check(lib().hpmdr_ctx_profile(self._p, int(enable)), "hpmdr_ctx_profile")
            return
        names = self.stage_names()
        mask = 0
        for nm in stages:
            mask |= 1 << names.index(nm)
        _check(lib().hpmdr_ctx_profile_stages(self._p, mask if enable else 0),
               "hpmdr_ctx_profile_stages")

    def stage_names(self):
        out, i = [], 0
        while True:
            name, ms, calls, by = C.c_char_p(), C.c_double(), C.c_uint64(), C.c_double()
            if lib().hpmdr_ctx_profile_entry(self._p, i, C.byref(name), C.byref(ms), C.byref(calls),
                                             C.byref(by)) != OK:
                return out
            out.append(name.value.decode())
            i += 1

    def profile_entries(self):
        """[(stage name, total ms, launches, algorithmic bytes)] since profile(True)."""
        out = []
        i = 0
        while True:
            name, ms, calls, by = C.c_char_p(), C.c_double(), C.c_uint64(), C.c_double()
            st = lib().hpmdr_ctx_profile_entry(self._p, i, C.byref(name), C.byref(ms), C.byref(calls),
                                               C.byref(by))
            if st != OK:
                break
            out.append((name.value.decode(), ms.value, calls.value, by.value))
            i += 1
        return out

    def set_stream(self, stream):
        _check(lib().hpmdr_ctx_set_stream(self._p, _stream_ptr(stream)), "hpmdr_ctx_set_stream")

    def close(self):
        if self._p:
            lib().hpmdr_ctx_destroy(self._p)
            self._p = vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- refactor / retrieve ------------------------------------------------
    def refactor(self, field):
        """field: torch tensor (CUDA or CPU), float32/float64, 1-3 dims, contiguous."""
        import torch
        if not field.is_contiguous():
            raise ValueError("field must be contiguous")
        nd, dims = _dims3(field.shape)
        out = vp()
        _check(lib().hpmdr_refactor(self._p, vp(field.data_ptr()), int(field.is_cuda), nd, dims,
                                    _dtype_code(field), C.byref(out)), "hpmdr_refactor")
        return Handle(self, out, tuple(field.shape), field.dtype)

    def import_handle(self, blob):
        buf = (C.c_uint8 * len(blob)).from_buffer_copy(bytes(blob))
        out = vp()
        _check(lib().hpmdr_handle_import(self._p, buf, len(blob), C.byref(out)), "hpmdr_handle_import")
        h = Handle(self, out, None, None)
        h._fill_shape()
        return h

    def retrieve_qoi_vmag(self, handles, rel_bound, outs=None, out_vmag=None):
        """handles: three FP32 Handles; outs: three tensors or None; returns (vmag, infos)."""
        import torch
        ref = handles[0]
        dev = outs[0].is_cuda if outs is not None and outs[0] is not None else True
        if out_vmag is None:
            out_vmag = torch.empty(ref.shape, dtype=torch.float32,
                                   device="cuda" if dev else "cpu")
        arr = (vp * 3)(*[h._p for h in handles])
        oarr = (vp * 3)(*[(vp(o.data_ptr()) if o is not None else None) for o in (outs or [None] * 3)])
        infos = (RetrieveInfo * 4)()
        st = lib().hpmdr_retrieve_qoi_vmag(self._p, arr, float(rel_bound), oarr,
                                           vp(out_vmag.data_ptr()), int(out_vmag.is_cuda), infos)
        _check(st, "hpmdr_retrieve_qoi_vmag", allow=(ERR_UNATTAINABLE,))
        return out_vmag, list(infos), st

    def refactor_chunked(self, field, chunk, nstreams=2):
        """Refactor `field` (contiguous tensor, pinned CPU or CUDA) as independent
        chunks of shape `chunk`; returns the chunk handles in C order."""
        if not field.is_contiguous():
            raise ValueError("field must be contiguous")
        nd, dims = _dims3(field.shape)
        ndc, cdims = _dims3(chunk)
        if ndc != nd:
            raise ValueError("chunk needs as many dimensions as the field")
        n = C.c_uint64()
        _check(lib().hpmdr_refactor_chunked(self._p, None, 0, nd, dims, cdims, _dtype_code(field), 1,
                                            None, 0, C.byref(n)), "hpmdr_refactor_chunked")
        arr = (vp * n.value)()
        _check(lib().hpmdr_refactor_chunked(self._p, vp(field.data_ptr()), int(field.is_cuda), nd,
                                            dims, cdims, _dtype_code(field), int(nstreams), arr,
                                            n.value, C.byref(n)), "hpmdr_refactor_chunked")
        out = []
        for i in range(n.value):
            h = Handle(self, vp(arr[i]), None, None)
            h._fill_shape()
            out.append(h)
        return out

    def retrieve_chunked(self, handles, shape, chunk, rel_bound, out, nstreams=2):
        """Reconstruct a chunk-streamed field into `out` (tensor of `shape`);
        returns (infos, status)."""
        nd, dims = _dims3(shape)
        _, cdims = _dims3(chunk)
        arr = (vp * len(handles))(*[h._p for h in handles])
        infos = (RetrieveInfo * len(handles))()
        st = lib().hpmdr_retrieve_chunked(self._p, arr, len(handles), nd, dims, cdims,
                                          float(rel_bound), vp(out.data_ptr()), int(out.is_cuda),
                                          int(nstreams), infos)
        _check(st, "hpmdr_retrieve_chunked", allow=(ERR_UNATTAINABLE,))
        return list(infos), st

    def prepare_vtotal(self, handles, vx, vy, vz):
        arr = (vp * 3)(*[h._p for h in handles])
        _check(lib().hpmdr_qoi_prepare_vtotal(self._p, arr, vp(vx.data_ptr()), vp(vy.data_ptr()),
                                              vp(vz.data_ptr()), int(vx.is_cuda)),
               "hpmdr_qoi_prepare_vtotal")

    def retrieve_qoi_vtotal(self, handles, rel_bound, estimator, c=0.0, outs=None, out_q=None):
        """Algorithm 3 for V = vx^2+vy^2+vz^2; returns (V_hat, report, status)."""
        import torch
        ref = handles[0]
        if out_q is None:
            out_q = torch.empty(ref.shape, dtype=torch.float32, device="cuda")
        arr = (vp * 3)(*[h._p for h in handles])
        oarr = (vp * 3)(*[(vp(o.data_ptr()) if o is not None else None) for o in (outs or [None] * 3)])
        rep = QoiReport()
        st = lib().hpmdr_retrieve_qoi_vtotal(self._p, arr, float(rel_bound), int(estimator), float(c),
                                             oarr, vp(out_q.data_ptr()), int(out_q.is_cuda),
                                             C.byref(rep))
        _check(st, "hpmdr_retrieve_qoi_vtotal", allow=(ERR_UNATTAINABLE,))
        return out_q, rep, st

    def prepare_vmag(self, handles, vx, vy, vz):
        arr = (vp * 3)(*[h._p for h in handles])
        _check(lib().hpmdr_qoi_prepare_vmag(self._p, arr, vp(vx.data_ptr()), vp(vy.data_ptr()),
                                            vp(vz.data_ptr()), int(vx.is_cuda)),
               "hpmdr_qoi_prepare_vmag")

    # ---- stage entry points ---------------------------------------------------
    def encode_group(self, G, force=-1, cap=None):
        import torch
        cap = cap if cap is not None else G.numel() * 2 + 4096
        out = torch.empty(cap, dtype=torch.uint8, device=G.device)
        ln, m = C.c_uint64(0), C.c_int(0)
        _check(lib().hpmdr_encode_group(self._p, vp(G.data_ptr()), G.numel(), force,
                                        vp(out.data_ptr()), cap, C.byref(ln), C.byref(m)),
               "hpmdr_encode_group")
        return out[: ln.value], m.value

    def decode_group(self, data, method, S):
        import torch
        G = torch.empty(S, dtype=torch.uint8, device=data.device)
        st = lib().hpmdr_decode_group(self._p, vp(data.data_ptr()), data.numel(), method,
                                      vp(G.data_ptr()), S)
        return st, G


    def fixed_to_float(self, X, E_f, dtype):
        """RN(X) * 2^(E_f - 48) in dtype for a device int64 tensor X (the output
        conversion of every retrieval)."""
        import torch
        out = torch.empty(X.shape, dtype=dtype, device=X.device)
        _check(lib().hpmdr_fixed_to_float(self._p, vp(X.data_ptr()), X.numel(), E_f,
                                          F32 if dtype == torch.float32 else F64,
                                          vp(out.data_ptr())), "hpmdr_fixed_to_float")
        return out


    def vtotal_bound(self, vx, vy, vz, e):
        """One QoI bounding step on three device FP32 tensors of one shape:
        (V_hat, largest pointwise bound, its first point)."""
        import torch
        out = torch.empty(vx.shape, dtype=torch.float32, device=vx.device)
        b, pt = C.c_double(), C.c_uint64()
        _check(lib().hpmdr_qoi_vtotal_bound(self._p, vp(vx.data_ptr()), vp(vy.data_ptr()),
                                            vp(vz.data_ptr()), vx.numel(),
                                            (C.c_double * 3)(*[float(x) for x in e]),
                                            vp(out.data_ptr()), C.byref(b), C.byref(pt)),
               "hpmdr_qoi_vtotal_bound")
        return out, b.value, pt.value


class Handle:
    """One refactored field (hpmdr_handle) and its incremental retrieval state."""

    def __init__(self, ctx, p, shape, dtype):
        self.ctx, self._p, self.shape, self.dtype = ctx, p, shape, dtype

    def _fill_shape(self):
        import torch
        info = self.field_info()
        self.shape = tuple(int(d) for d in info["dims"])
        self.dtype = torch.float32 if info["dtype"] == F32 else torch.float64

    def free(self):
        if self._p:
            lib().hpmdr_handle_free(self._p)
            self._p = vp()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def retrieve(self, bound, out=None, absolute=False):
        """Reconstruct into `out` (allocated on the GPU if None).  Returns (out, info, status)."""
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        info = RetrieveInfo()
        fn = lib().hpmdr_retrieve_abs if absolute else lib().hpmdr_retrieve
        st = fn(self.ctx._p, self._p, float(bound), vp(out.data_ptr()), int(out.is_cuda),
                C.byref(info))
        _check(st, "hpmdr_retrieve", allow=(ERR_UNATTAINABLE,))
        return out, info, st

    def retrieve_async(self, bound, out):
        """Enqueue a retrieval into `out` (a CUDA tensor, or page-locked host
        memory) without waiting; out and the returned info are complete at
        Context.wait()."""
        info = RetrieveInfo()
        self.ctx._keep.append((info, out))
        fn = lib().hpmdr_retrieve_async if out.is_cuda else lib().hpmdr_retrieve_async_host
        _check(fn(self.ctx._p, self._p, float(bound), vp(out.data_ptr()), C.byref(info)),
               "hpmdr_retrieve_async")
        return info

    def field_info(self):
        dt, nl, ef, ie = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        dims = (C.c_uint64 * 3)()
        stats = (C.c_double * 4)()
        _check(lib().hpmdr_handle_field_info(self._p, C.byref(dt), dims, C.byref(nl), C.byref(ef),
                                             C.byref(ie), stats), "hpmdr_handle_field_info")
        return {"dtype": dt.value, "dims": list(dims), "nlevels": nl.value, "E_f": ef.value,
                "input_exact": bool(ie.value), "maxabs": stats[0], "vmin": stats[1],
                "vmax": stats[2], "range": stats[3]}

    def level_info(self, level):
        n, bl, ng, ex = C.c_uint64(), C.c_int(), C.c_int(), C.c_int()
        _check(lib().hpmdr_handle_level_info(self._p, level, C.byref(n), C.byref(bl), C.byref(ng),
                                             C.byref(ex)), "hpmdr_handle_level_info")
        return n.value, bl.value, ng.value, bool(ex.value)

    def group(self, level, group):
        """(stored bytes as a numpy uint8 array, method, (est_H, est_R))"""
        import numpy as np
        ln, m = C.c_uint64(), C.c_int()
        est = (C.c_uint64 * 2)()
        _check(lib().hpmdr_handle_group(self._p, level, group, None, C.byref(ln), C.byref(m), est),
               "hpmdr_handle_group")
        buf = np.zeros(ln.value, dtype=np.uint8)
        _check(lib().hpmdr_handle_group(self._p, level, group, buf.ctypes.data_as(vp), C.byref(ln),
                                        C.byref(m), est), "hpmdr_handle_group")
        return buf, m.value, (int(est[0]), int(est[1]))

    def planes(self, level):
        import numpy as np
        ln = C.c_uint64()
        _check(lib().hpmdr_handle_planes(self._p, level, None, C.byref(ln)), "hpmdr_handle_planes")
        buf = np.zeros(ln.value // 4, dtype=np.uint32)
        _check(lib().hpmdr_handle_planes(self._p, level, buf.ctypes.data_as(vp), C.byref(ln)),
               "hpmdr_handle_planes")
        return buf

    def sequence(self):
        n = C.c_int()
        _check(lib().hpmdr_handle_sequence(self._p, None, 0, C.byref(n)), "hpmdr_handle_sequence")
        arr = (C.c_int * max(n.value, 1))()
        _check(lib().hpmdr_handle_sequence(self._p, arr, n.value, C.byref(n)), "hpmdr_handle_sequence")
        return list(arr[: n.value])

    def export(self):
        ln = C.c_uint64()
        _check(lib().hpmdr_handle_export(self._p, None, C.byref(ln)), "hpmdr_handle_export")
        buf = (C.c_uint8 * ln.value)()
        _check(lib().hpmdr_handle_export(self._p, buf, C.byref(ln)), "hpmdr_handle_export")
        return bytes(buf)

    def reset(self, poison=False):
        _check(lib().hpmdr_handle_reset(self.ctx._p, self._p, int(poison)), "hpmdr_handle_reset")

    def compact(self):
        _check(lib().hpmdr_handle_compact(self.ctx._p, self._p), "hpmdr_handle_compact")

    def drop_cache(self):
        _check(lib().hpmdr_handle_drop_cache(self.ctx._p, self._p), "hpmdr_handle_drop_cache")

    def memory(self):
        """(resident, cache, cache_max) device bytes"""
        r, c, m = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(lib().hpmdr_handle_memory(self._p, C.byref(r), C.byref(c), C.byref(m)),
               "hpmdr_handle_memory")
        return r.value, c.value, m.value


def bitplane_encode(q, sign, B, stream=None):
    """q: CUDA int32/int64 tensor viewed as uint32/uint64 bits; sign: uint8 tensor."""
    import torch
    n = q.numel()
    W = 4 * ((n + 127) // 128)
    planes = torch.empty((B + 1) * W, dtype=torch.int32, device=q.device)
    _check(lib().hpmdr_bitplane_encode(vp(q.data_ptr()), vp(sign.data_ptr()), n, B,
                                       vp(planes.data_ptr()), _stream_ptr(stream)),
           "hpmdr_bitplane_encode")
    return planes


def bitplane_decode(planes, n, B, k, stream=None):
    import torch
    q = torch.empty(n, dtype=torch.int32 if B == 32 else torch.int64, device=planes.device)
    s = torch.empty(n, dtype=torch.uint8, device=planes.device)
    _check(lib().hpmdr_bitplane_decode(vp(planes.data_ptr()), n, B, k, vp(q.data_ptr()),
                                       vp(s.data_ptr()), _stream_ptr(stream)),
           "hpmdr_bitplane_decode")
    return q, s


BP_REGISTER_BLOCK, BP_LOCALITY_BLOCK, BP_SHUFFLE_BALLOT, BP_SHUFFLE_SHIFT, \
    BP_SHUFFLE_MATCH_ANY, BP_SHUFFLE_REDUCE = range(6)
BP_DESIGNS = {"register_block": 0, "locality_block": 1, "shuffle_ballot": 2, "shuffle_shift": 3,
              "shuffle_match_any": 4, "shuffle_reduce": 5}


def bitplane_encode_design(q, sign, design, planes=None, stream=None):
    """One of the Sec. 4 encoder designs (B = 32) on a CUDA int32 tensor q."""
    import torch
    n = q.numel()
    W = 4 * ((n + 127) // 128)
    if planes is None:
        planes = torch.empty(33 * W, dtype=torch.int32, device=q.device)
    _check(lib().hpmdr_bitplane_encode_design(vp(q.data_ptr()), vp(sign.data_ptr()), n, design,
                                              vp(planes.data_ptr()), _stream_ptr(stream)),
           "hpmdr_bitplane_encode_design")
    return planes


def bitplane_decode_design(planes, n, design, k, q=None, sign=None, stream=None):
    import torch
    if q is None:
        q = torch.empty(n, dtype=torch.int32, device=planes.device)
    if sign is None:
        sign = torch.empty(n, dtype=torch.uint8, device=planes.device)
    _check(lib().hpmdr_bitplane_decode_design(vp(planes.data_ptr()), n, design, k,
                                              vp(q.data_ptr()), vp(sign.data_ptr()),
                                              _stream_ptr(stream)),
           "hpmdr_bitplane_decode_design")
    return q, sign


class Server:
    """hpmdr_server: concurrent retrieval requests over added handles."""

    def __init__(self, ctx, hbm_budget, max_slots=8, keep_cache=True, queue_timeout_s=0.0):
        self.ctx = ctx
        cfg = ServerConfig(int(max_slots), int(bool(keep_cache)), int(hbm_budget),
                           float(queue_timeout_s))
        self._p = vp()
        _check(lib().hpmdr_server_create(ctx._p, C.byref(cfg), C.byref(self._p)),
               "hpmdr_server_create")
        self._keep = {}

    def add(self, handle):
        _check(lib().hpmdr_server_add_field(self._p, self.ctx._p, handle._p), "hpmdr_server_add_field")

    def submit(self, handles, rel_bound, out=None, out_vmag=None):
        """One handle: field request into `out`; three handles: |v| into `out_vmag`
        (out: optional list of three component tensors).  Returns the ticket."""
        r = Request()
        if len(handles) == 1:
            r.kind = REQ_FIELD
            r.h[0] = handles[0]._p
            r.out[0] = out.data_ptr()
            keep = (out,)
        else:
            r.kind = REQ_VMAG
            for i in range(3):
                r.h[i] = handles[i]._p
                r.out[i] = out[i].data_ptr() if out is not None and out[i] is not None else None
            r.out_vmag = out_vmag.data_ptr()
            keep = (out, out_vmag)
        r.rel_bound = float(rel_bound)
        t = C.c_uint64()
        _check(lib().hpmdr_server_submit(self._p, C.byref(r), C.byref(t)), "hpmdr_server_submit")
        self._keep[t.value] = keep
        return t.value

    def poll(self, ticket, wait=True):
        """(status, infos, (t_submit, t_start, t_done)) or None while pending."""
        infos = (RetrieveInfo * 4)()
        times = (C.c_double * 3)()
        st = lib().hpmdr_server_poll(self._p, ticket, int(wait), infos, times)
        if st == ERR_BUSY:
            return None
        self._keep.pop(ticket, None)
        _check(st, "hpmdr_server_poll", allow=(ERR_UNATTAINABLE, ERR_TIMEOUT, ERR_CANCELLED))
        return st, list(infos), tuple(times)

    def cancel(self, ticket):
        """True if the request was still queued and is now cancelled (its poll
        returns ERR_CANCELLED); False if it has started or finished."""
        st = lib().hpmdr_server_cancel(self._p, ticket)
        if st == ERR_BUSY:
            return False
        _check(st, "hpmdr_server_cancel")
        return True

    def stats(self):
        a = (C.c_uint64 * 6)()
        _check(lib().hpmdr_server_stats(self._p, a), "hpmdr_server_stats")
        return dict(zip(["used", "peak", "evictions", "completed", "queued", "running"], list(a)))

    def close(self):
        if self._p:
            lib().hpmdr_server_destroy(self._p)
            self._p = vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BorrowedHandle(Handle):
    """A handle owned by a Batch (never freed from Python)."""

    def free(self):
        self._p = vp()


class Batch:
    """hpmdr_batch: many fields refactored / retrieved by one graph launch per pass."""

    def __init__(self, ctx, shapes, dtype):
        import torch
        self.ctx = ctx
        self.shapes = [tuple(int(d) for d in ((1,) * (3 - len(sh)) + tuple(sh))) for sh in shapes]
        self.dtype = dtype
        n = len(self.shapes)
        dims = (C.c_uint64 * (3 * n))(*[d for sh in self.shapes for d in sh])
        self._p = vp()
        code = F32 if dtype == torch.float32 else F64
        _check(lib().hpmdr_batch_create(ctx._p, n, dims, code, C.byref(self._p)), "hpmdr_batch_create")
        self.handles = []
        for i in range(n):
            h = vp()
            _check(lib().hpmdr_batch_handle(self._p, i, C.byref(h)), "hpmdr_batch_handle")
            self.handles.append(BorrowedHandle(ctx, h, self.shapes[i], dtype))

    def _ptrs(self, tensors):
        return (vp * len(tensors))(*[t.data_ptr() for t in tensors])

    def refactor(self, fields):
        _check(lib().hpmdr_batch_refactor(self._p, self._ptrs(fields)), "hpmdr_batch_refactor")

    def retrieve(self, bounds, outs):
        n = len(self.shapes)
        b = (C.c_double * n)(*[float(x) for x in bounds])
        infos = (RetrieveInfo * n)()
        st = lib().hpmdr_batch_retrieve(self._p, b, self._ptrs(outs), infos)
        _check(st, "hpmdr_batch_retrieve", allow=(ERR_UNATTAINABLE,))
        return list(infos), st

    def autotune(self, fields, bounds, outs):
        n = len(self.shapes)
        b = (C.c_double * n)(*[float(x) for x in bounds])
        best = (C.c_uint32 * 3)()
        _check(lib().hpmdr_batch_autotune(self._p, self._ptrs(fields), b, self._ptrs(outs), best),
               "hpmdr_batch_autotune")
        return tuple(best)

    def set_tuning(self, grid_mul, seg, dec_mul):
        _check(lib().hpmdr_batch_set_tuning(self._p, (C.c_uint32 * 3)(grid_mul, seg, dec_mul)),
               "hpmdr_batch_set_tuning")

    def tuning(self):
        t = (C.c_uint32 * 3)()
        _check(lib().hpmdr_batch_get_tuning(self._p, t), "hpmdr_batch_get_tuning")
        return tuple(t)

    def last_ms(self):
        ms = (C.c_double * 2)()
        _check(lib().hpmdr_batch_last_ms(self._p, ms), "hpmdr_batch_last_ms")
        return ms[0], ms[1]

    def close(self):
        for h in self.handles:
            h._p = vp()
        if self._p:
            lib().hpmdr_batch_destroy(self._p)
            self._p = vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
