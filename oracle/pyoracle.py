"""ctypes view of the CPU oracle (test infrastructure only).

Marshals numpy arrays into the plain C oracle in ``oracle/*.c``.  The product
package never imports this module.
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None

OR_F32, OR_F64 = 0, 1
DC, HUFFMAN, RLE, PLACEHOLDER = 0, 1, 2, 3
OK, ERR_ARG, ERR_CORRUPT, ERR_UNATTAINABLE = 0, -1, -4, -5
CHUNK = 16384

u64p = C.POINTER(C.c_uint64)
dims_t = C.c_uint64 * 3


class HybridCfg(C.Structure):
    _fields_ = [("Ts", C.c_uint64), ("cr_num", C.c_uint32), ("cr_den", C.c_uint32)]


class SelMeta(C.Structure):
    _fields_ = [("nlev", C.c_int), ("B", C.c_int), ("dtype", C.c_int), ("E_f", C.c_int),
                ("input_exact", C.c_int), ("bl", C.c_int * 64), ("exact", C.c_int * 64),
                ("ngroups", C.c_int * 64), ("group_bytes", u64p * 64)]


class Stats(C.Structure):
    _fields_ = [("maxabs", C.c_double), ("vmin", C.c_double), ("vmax", C.c_double),
                ("range", C.c_double), ("E_f", C.c_int), ("input_exact", C.c_int)]


class QoiReport(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("tau_abs", C.c_double),
                ("est", C.c_double), ("eps", C.c_double * 3), ("prefix", C.c_int * 3),
                ("g", (C.c_int * 64) * 3)]


EST_CP, EST_MA, EST_MAPE = 0, 1, 2


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        vp, cvp = C.c_void_p, C.c_void_p
        sig = {
            "or_num_levels": (C.c_int, [dims_t]),
            "or_level_size": (C.c_uint64, [dims_t, C.c_int]),
            "or_plane_words": (C.c_uint64, [C.c_uint64]),
            "or_field_stats": (C.c_int, [cvp, C.c_uint64, C.c_int, C.POINTER(Stats)]),
            "or_fixed_point": (C.c_int64, [cvp, C.c_uint64, C.c_int, C.c_int, C.POINTER(C.c_int)]),
            "or_level_coeffs": (None, [cvp, dims_t, C.c_int, C.c_int, C.c_int, vp]),
            "or_bitlen_max": (C.c_int, [vp, C.c_uint64]),
            "or_quantize": (None, [vp, C.c_uint64, C.c_int, C.c_int, vp, vp]),
            "or_level_exact": (C.c_int, [vp, C.c_uint64, C.c_int, C.c_int]),
            "or_bitplane_encode": (None, [vp, vp, C.c_uint64, C.c_int, vp]),
            "or_bitplane_decode": (None, [vp, C.c_uint64, C.c_int, C.c_int, vp, vp]),
            "or_num_groups": (C.c_int, [C.c_int]),
            "or_group_offset": (C.c_uint64, [C.c_uint64, C.c_int]),
            "or_group_size": (C.c_uint64, [C.c_uint64, C.c_int]),
            "or_histogram": (None, [vp, C.c_uint64, vp]),
            "or_huffman_lengths": (None, [vp, vp]),
            "or_huffman_estimate": (C.c_uint64, [vp, vp, C.c_uint64]),
            "or_huffman_encode": (C.c_uint64, [vp, C.c_uint64, vp]),
            "or_huffman_decode": (C.c_int, [vp, C.c_uint64, vp, C.c_uint64]),
            "or_rle_estimate": (C.c_uint64, [vp, C.c_uint64]),
            "or_rle_encode": (C.c_uint64, [vp, C.c_uint64, vp]),
            "or_rle_decode": (C.c_int, [vp, C.c_uint64, vp, C.c_uint64]),
            "or_hybrid_choose": (C.c_int, [C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(HybridCfg)]),
            "or_hybrid_encode": (C.c_uint64, [vp, C.c_uint64, C.POINTER(HybridCfg), C.POINTER(C.c_int), vp]),
            "or_estimate": (None, [C.POINTER(SelMeta), vp, u64p, u64p]),
            "or_greedy_sequence": (C.c_int, [C.POINTER(SelMeta), vp, C.c_int]),
            "or_select": (C.c_int, [C.POINTER(SelMeta), C.c_double, vp, C.POINTER(C.c_double), u64p, u64p]),
            "or_units_to_abs": (C.c_double, [C.c_uint64, C.c_uint64, C.c_int, C.c_int]),
            "or_tau_units": (None, [C.c_double, C.c_int, C.c_int, u64p, u64p]),
            "or_recompose": (None, [dims_t, C.c_int, C.c_int, vp, vp]),
            "or_dequantize": (C.c_int64, [C.c_uint64, C.c_int, C.c_int, C.c_int]),
            "or_vmag": (C.c_float, [C.c_float, C.c_float, C.c_float]),
            "or_vmag_field": (None, [vp, vp, vp, C.c_uint64, vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
            "or_qoi_component_bound": (C.c_double, [C.c_double, C.c_double]),
            "or_qoi_estimate": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_double]),
            "or_refactor": (vp, [cvp, dims_t, C.c_int, C.POINTER(HybridCfg), C.POINTER(C.c_int)]),
            "or_field_free": (None, [vp]),
            "or_field_select": (C.c_int, [vp, C.c_double, vp, C.POINTER(C.c_double), u64p, u64p]),
            "or_field_sequence": (C.c_int, [vp, vp, C.c_int]),
            "or_reconstruct": (C.c_int, [vp, vp, vp]),
            "or_retrieve": (C.c_int, [vp, C.c_double, vp, vp, C.POINTER(C.c_double), u64p, u64p]),
            "or_field_info": (None, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), vp]),
            "or_field_level": (None, [vp, C.c_int, u64p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "or_field_planes": (vp, [vp, C.c_int]),
            "or_field_group": (vp, [vp, C.c_int, C.c_int, u64p, C.POINTER(C.c_int), vp]),
            "or_field_estimate": (None, [vp, vp, C.POINTER(C.c_double)]),
            "or_vtotal": (C.c_double, [C.c_float, C.c_float, C.c_float]),
            "or_vtotal_range": (None, [vp, vp, vp, C.c_uint64, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]),
            "or_vtotal_point_bound": (C.c_double, [C.c_float, C.c_float, C.c_float, vp]),
            "or_vtotal_bound": (C.c_double, [vp, vp, vp, C.c_uint64, vp, u64p]),
            "or_field_prefix_estimate": (C.c_double, [vp, C.c_int]),
            "or_qoi_vtotal": (C.c_int, [vp, C.c_uint64, C.c_double, C.c_double, C.c_double, C.c_int,
                                        C.c_double, vp, vp, C.POINTER(QoiReport)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _dims(shape):
    s = tuple(int(x) for x in shape)
    s = (1,) * (3 - len(s)) + s
    return dims_t(*s)


def _dtype_code(a):
    if a.dtype == np.float32:
        return OR_F32
    if a.dtype == np.float64:
        return OR_F64
    raise TypeError(a.dtype)


# ---------------------------------------------------------------- steps
def num_levels(shape):
    return lib().or_num_levels(_dims(shape))


def level_size(shape, l):
    return int(lib().or_level_size(_dims(shape), l))


def plane_words(n):
    return int(lib().or_plane_words(n))


def field_stats(f):
    f = np.ascontiguousarray(f)
    st = Stats()
    rc = lib().or_field_stats(_p(f), f.size, _dtype_code(f), C.byref(st))
    return rc, st


def fixed_point(f, i, E_f):
    f = np.ascontiguousarray(f)
    fl = C.c_int(0)
    v = lib().or_fixed_point(_p(f), i, _dtype_code(f), E_f, C.byref(fl))
    return int(v), bool(fl.value)


def level_coeffs(f, E_f, l):
    f = np.ascontiguousarray(f)
    n = level_size(f.shape, l)
    out = np.zeros(n, dtype=np.int64)
    lib().or_level_coeffs(_p(f), _dims(f.shape), _dtype_code(f), E_f, l, _p(out))
    return out


def bitlen_max(C8):
    C8 = np.ascontiguousarray(C8, dtype=np.int64)
    return lib().or_bitlen_max(_p(C8), C8.size)


def quantize(C8, B, bl):
    C8 = np.ascontiguousarray(C8, dtype=np.int64)
    q = np.zeros(C8.size, dtype=np.uint64)
    s = np.zeros(C8.size, dtype=np.uint8)
    lib().or_quantize(_p(C8), C8.size, B, bl, _p(q), _p(s))
    return q, s


def level_exact(C8, B, bl):
    C8 = np.ascontiguousarray(C8, dtype=np.int64)
    return bool(lib().or_level_exact(_p(C8), C8.size, B, bl))


def bitplane_encode(q, sign, B):
    q = np.ascontiguousarray(q, dtype=np.uint64)
    sign = np.ascontiguousarray(sign, dtype=np.uint8)
    W = plane_words(q.size)
    planes = np.zeros((B + 1) * W, dtype=np.uint32)
    lib().or_bitplane_encode(_p(q), _p(sign), q.size, B, _p(planes))
    return planes.reshape(B + 1, W)


def bitplane_decode(planes, n, B, k):
    planes = np.ascontiguousarray(planes, dtype=np.uint32)
    q = np.zeros(n, dtype=np.uint64)
    s = np.zeros(n, dtype=np.uint8)
    lib().or_bitplane_decode(_p(planes), n, B, k, _p(q), _p(s))
    return q, s


def dequantize(qhat, s, B, bl):
    return int(lib().or_dequantize(int(qhat), int(s), B, bl))


def group_slice(W, g):
    return int(lib().or_group_offset(W, g)), int(lib().or_group_size(W, g))


def histogram(G):
    G = np.ascontiguousarray(G, dtype=np.uint8)
    h = np.zeros(256, dtype=np.uint64)
    lib().or_histogram(_p(G), G.size, _p(h))
    return h


def huffman_lengths(hist):
    hist = np.ascontiguousarray(hist, dtype=np.uint64)
    ln = np.zeros(256, dtype=np.uint8)
    lib().or_huffman_lengths(_p(hist), _p(ln))
    return ln


def huffman_estimate(hist, lens, S):
    hist = np.ascontiguousarray(hist, dtype=np.uint64)
    lens = np.ascontiguousarray(lens, dtype=np.uint8)
    return int(lib().or_huffman_estimate(_p(hist), _p(lens), S))


def _encode(fn, G):
    G = np.ascontiguousarray(G, dtype=np.uint8)
    n = fn(_p(G), G.size, None)
    out = np.zeros(n, dtype=np.uint8)
    fn(_p(G), G.size, _p(out))
    return out


def huffman_encode(G):
    return _encode(lib().or_huffman_encode, G)


def rle_encode(G):
    return _encode(lib().or_rle_encode, G)


def _decode(fn, data, S):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    G = np.zeros(S, dtype=np.uint8)
    rc = fn(_p(data), data.size, _p(G), S)
    return rc, G


def huffman_decode(data, S):
    return _decode(lib().or_huffman_decode, data, S)


def rle_decode(data, S):
    return _decode(lib().or_rle_decode, data, S)


def rle_estimate(G):
    G = np.ascontiguousarray(G, dtype=np.uint8)
    return int(lib().or_rle_estimate(_p(G), G.size))


def hybrid_cfg(Ts=4096, cr_num=2, cr_den=1):
    return HybridCfg(Ts, cr_num, cr_den)


def hybrid_encode(G, Ts=4096, cr_num=2, cr_den=1):
    G = np.ascontiguousarray(G, dtype=np.uint8)
    cfg = hybrid_cfg(Ts, cr_num, cr_den)
    m = C.c_int()
    n = lib().or_hybrid_encode(_p(G), G.size, C.byref(cfg), C.byref(m), None)
    out = np.zeros(n, dtype=np.uint8)
    lib().or_hybrid_encode(_p(G), G.size, C.byref(cfg), C.byref(m), _p(out))
    return out, m.value


def hybrid_choose(S, est_H, est_R, cfg=None):
    cfg = cfg or hybrid_cfg()
    return lib().or_hybrid_choose(S, est_H, est_R, C.byref(cfg))


def tau_units(tau_abs, E_f, B):
    hi, lo = C.c_uint64(), C.c_uint64()
    lib().or_tau_units(tau_abs, E_f, B, C.byref(hi), C.byref(lo))
    return (hi.value << 64) | lo.value


def units_to_abs(E, E_f, B):
    return lib().or_units_to_abs(E >> 64, E & ((1 << 64) - 1), E_f, B)


def make_meta(nlev, B, dtype, E_f, input_exact, bl, exact, group_bytes):
    """group_bytes: list (per level) of uint64 arrays; kept alive by the caller."""
    m = SelMeta()
    m.nlev, m.B, m.dtype, m.E_f, m.input_exact = nlev, B, dtype, E_f, int(input_exact)
    keep = []
    for l in range(nlev):
        m.bl[l] = int(bl[l])
        m.exact[l] = int(exact[l])
        gb = np.ascontiguousarray(group_bytes[l], dtype=np.uint64)
        keep.append(gb)
        m.ngroups[l] = gb.size
        m.group_bytes[l] = gb.ctypes.data_as(u64p)
    m._keep = keep
    return m


def estimate(meta, g):
    g = np.ascontiguousarray(g, dtype=np.int32)
    hi, lo = C.c_uint64(), C.c_uint64()
    lib().or_estimate(C.byref(meta), _p(g), C.byref(hi), C.byref(lo))
    return (hi.value << 64) | lo.value


def greedy_sequence(meta, cap=1024):
    seq = np.zeros(cap, dtype=np.int32)
    n = lib().or_greedy_sequence(C.byref(meta), _p(seq), cap)
    return seq[:n].tolist()


def select(meta, tau_abs):
    g = np.zeros(meta.nlev, dtype=np.int32)
    E = C.c_double()
    hi, lo = C.c_uint64(), C.c_uint64()
    rc = lib().or_select(C.byref(meta), tau_abs, _p(g), C.byref(E), C.byref(hi), C.byref(lo))
    return rc, g, E.value, (hi.value << 64) | lo.value


def recompose(shape, dtype_code, E_f, c8hats):
    """c8hats: list over levels of int64 arrays (or None for all-zero levels)."""
    nlev = len(c8hats)
    arrs = (C.c_void_p * nlev)()
    keep = []
    for l, a in enumerate(c8hats):
        if a is None:
            arrs[l] = None
        else:
            a = np.ascontiguousarray(a, dtype=np.int64)
            keep.append(a)
            arrs[l] = a.ctypes.data
    out = np.zeros(int(np.prod(shape)), dtype=np.float32 if dtype_code == OR_F32 else np.float64)
    lib().or_recompose(_dims(shape), dtype_code, E_f, arrs, _p(out))
    return out.reshape(shape)


def vmag(x, y, z):
    return lib().or_vmag(x, y, z)


def vmag_field(vx, vy, vz):
    vx, vy, vz = (np.ascontiguousarray(a, dtype=np.float32) for a in (vx, vy, vz))
    out = np.zeros(vx.shape, dtype=np.float32)
    lo, hi = C.c_float(), C.c_float()
    lib().or_vmag_field(_p(vx), _p(vy), _p(vz), vx.size, _p(out), C.byref(lo), C.byref(hi))
    return out, lo.value, hi.value


def qoi_component_bound(tau_q_abs, qmax):
    return lib().or_qoi_component_bound(tau_q_abs, qmax)


def qoi_estimate(Ex, Ey, Ez, qmax):
    return lib().or_qoi_estimate(Ex, Ey, Ez, qmax)


# ---------------------------------------------------------------- end to end
class Field:
    """Refactored field held by the oracle (stored bytes per group + metadata)."""

    def __init__(self, f, Ts=4096, cr_num=2, cr_den=1):
        self.f = np.ascontiguousarray(f)
        self.shape = self.f.shape
        self.dtype_code = _dtype_code(self.f)
        self.B = 32 if self.dtype_code == OR_F32 else 64
        self.cfg = hybrid_cfg(Ts, cr_num, cr_den)
        st = C.c_int(0)
        self._h = lib().or_refactor(_p(self.f), _dims(self.shape), self.dtype_code,
                                    C.byref(self.cfg), C.byref(st))
        self.status = st.value
        if not self._h:
            raise ValueError(f"oracle refactor failed: {self.status}")
        nlev, E_f, ie = C.c_int(), C.c_int(), C.c_int()
        stats = (C.c_double * 4)()
        lib().or_field_info(self._h, C.byref(nlev), C.byref(E_f), C.byref(ie), stats)
        self.nlev, self.E_f, self.input_exact = nlev.value, E_f.value, bool(ie.value)
        self.maxabs, self.vmin, self.vmax, self.range = list(stats)
        self.levels = []
        for l in range(self.nlev):
            n, bl, ex = C.c_uint64(), C.c_int(), C.c_int()
            lib().or_field_level(self._h, l, C.byref(n), C.byref(bl), C.byref(ex))
            self.levels.append((n.value, bl.value, bool(ex.value)))
        self.ngroups = self.B // 4

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_field_free(self._h)
            self._h = None

    def planes(self, l):
        n = self.levels[l][0]
        W = plane_words(n)
        ptr = lib().or_field_planes(self._h, l)
        arr = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(C.c_uint32)), shape=((self.B + 1) * W,))
        return arr.copy().reshape(self.B + 1, W)

    def group(self, l, g):
        ln, m = C.c_uint64(), C.c_int()
        est = (C.c_uint64 * 2)()
        ptr = lib().or_field_group(self._h, l, g, C.byref(ln), C.byref(m), est)
        data = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(C.c_uint8)), shape=(ln.value,)).copy()
        return data, m.value, int(est[0]), int(est[1])

    def group_sizes(self):
        return [[self.group(l, g)[0].size for g in range(self.ngroups)] for l in range(self.nlev)]

    def sequence(self):
        seq = np.zeros(self.nlev * 16 + 1, dtype=np.int32)
        n = lib().or_field_sequence(self._h, _p(seq), seq.size)
        return seq[:n].tolist()

    def select(self, tau_abs):
        g = np.zeros(self.nlev, dtype=np.int32)
        E = C.c_double()
        hi, lo = C.c_uint64(), C.c_uint64()
        rc = lib().or_field_select(self._h, tau_abs, _p(g), C.byref(E), C.byref(hi), C.byref(lo))
        return rc, g, E.value, (hi.value << 64) | lo.value

    def reconstruct(self, g):
        g = np.ascontiguousarray(g, dtype=np.int32)
        out = np.zeros(self.shape, dtype=self.f.dtype)
        rc = lib().or_reconstruct(self._h, _p(g), _p(out))
        return rc, out

    def retrieve(self, tau_abs):
        out = np.zeros(self.shape, dtype=self.f.dtype)
        g = np.zeros(self.nlev, dtype=np.int32)
        E = C.c_double()
        hi, lo = C.c_uint64(), C.c_uint64()
        rc = lib().or_retrieve(self._h, tau_abs, _p(out), _p(g), C.byref(E), C.byref(hi),
                               C.byref(lo))
        return rc, out, g, E.value


# ---------------------------------------------- QoI: total velocity, iterated
def vtotal(x, y, z):
    return float(lib().or_vtotal(float(x), float(y), float(z)))


def vtotal_range(vx, vy, vz):
    a = [np.ascontiguousarray(v, dtype=np.float32) for v in (vx, vy, vz)]
    lo, hi = C.c_double(), C.c_double()
    lib().or_vtotal_range(_p(a[0]), _p(a[1]), _p(a[2]), a[0].size, C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def vtotal_point_bound(x, y, z, e):
    ee = np.ascontiguousarray(e, dtype=np.float64)
    return float(lib().or_vtotal_point_bound(float(x), float(y), float(z), _p(ee)))


def vtotal_bound(x, y, z, e):
    a = [np.ascontiguousarray(v, dtype=np.float32) for v in (x, y, z)]
    ee = np.ascontiguousarray(e, dtype=np.float64)
    arg = C.c_uint64()
    b = lib().or_vtotal_bound(_p(a[0]), _p(a[1]), _p(a[2]), a[0].size, _p(ee), C.byref(arg))
    return float(b), int(arg.value)


def qoi_vtotal(fields, vt_min, vt_max, tau_rel, estimator, c=10.0):
    """Algorithm 3 for V = vx^2+vy^2+vz^2 over three oracle Fields (FP32).
    Returns (status, [x_hat, y_hat, z_hat], V_hat, report)."""
    F = (C.c_void_p * 3)(*[f._h for f in fields])
    shape = fields[0].shape
    outs = [np.zeros(shape, dtype=np.float32) for _ in range(3)]
    po = (C.c_void_p * 3)(*[o.ctypes.data for o in outs])
    q = np.zeros(shape, dtype=np.float32)
    rep = QoiReport()
    st = lib().or_qoi_vtotal(F, int(np.prod(shape)), float(vt_min), float(vt_max), float(tau_rel),
                             int(estimator), float(c), po, _p(q), C.byref(rep))
    return st, outs, q, rep
