"""GPU parity of the out-of-core pipeline (Sec. 5.3's refactoring and retrieval
pipelines): several variables in host memory, refactored chunk by chunk into
serialized streams in host memory on three queues, then retrieved back.

Every unit's stream must be byte-identical to exporting a plain refactor of
that chunk, and every retrieved box must equal, bit for bit, the oracle's
retrieval of that chunk at the absolute bound rel x (the variable's whole
range); the assembled field then meets that bound everywhere."""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2505_00227_gb300 import binding
    binding.lib()
    return binding


def _boxes(shape, chunk):
    cnt = [(s + c - 1) // c for s, c in zip(shape, chunk)]
    for iz in range(cnt[0]):
        for iy in range(cnt[1]):
            for ix in range(cnt[2]):
                org = (iz * chunk[0], iy * chunk[1], ix * chunk[2])
                yield tuple(slice(o, min(o + c, s)) for o, c, s in zip(org, chunk, shape))


def _vars(shape, dtype, seed):
    from paper_2505_00227_gb300 import synthetic as S
    return [S.spectral(shape, seed=seed, dtype=dtype).numpy(),
            S.blobs(shape, seed=seed + 1, dtype=dtype).numpy(),
            S.spectral_trend(shape, seed=seed + 2, dtype=dtype).numpy()]


CASES = {
    # FP32, ragged chunk grid on every axis, chunks whose x-extent takes the cell kernels
    "f32_ragged": ((40, 70, 150), (16, 32, 128), torch.float32),
    # FP64, two variables' chunks of one z-slab each
    "f64_slabs": ((12, 20, 33), (5, 20, 33), torch.float64),
}


@pytest.mark.parametrize("queues", [3, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_pipeline_streams_and_retrievals(B, name, queues):
    shape, chunk, dtype = CASES[name]
    fs = _vars(shape, dtype, 40)
    host = [torch.from_numpy(f).pin_memory() for f in fs]
    ctx = B.Context()
    streams, offs, sizes = ctx.refactor_pipeline(host, chunk, queues=queues)
    boxes = list(_boxes(shape, chunk))
    assert len(offs) == len(fs) * len(boxes)
    blob = streams.numpy()
    for v, f in enumerate(fs):
        for c, bx in enumerate(boxes):
            u = v * len(boxes) + c
            part = torch.from_numpy(np.ascontiguousarray(f[bx])).cuda()
            ref = ctx.refactor(part).export()
            assert offs[u] % 16 == 0 and sizes[u] == len(ref)
            assert blob[offs[u]: offs[u] + sizes[u]].tobytes() == ref, (v, c)
    for rels in ([1e-2, 1e-4, 1e-6], [1e-6, 1e-1, 1e-3]):
        outs = [torch.empty(shape, dtype=dtype).pin_memory() for _ in fs]
        infos, st = ctx.retrieve_pipeline(streams, offs, sizes, shape, chunk, rels, outs,
                                          queues=queues)
        worst = 0
        for v, (f, rel) in enumerate(zip(fs, rels)):
            tau = rel * (float(f.max()) - float(f.min()))
            got = outs[v].numpy()
            for c, bx in enumerate(boxes):
                Fc = O.Field(np.ascontiguousarray(f[bx]))
                rc, ref, g, E = Fc.retrieve(tau)
                info = infos[v * len(boxes) + c]
                assert info.status == rc and list(info.groups_per_level[:info.nlevels]) == list(g)
                assert np.array_equal(np.ascontiguousarray(got[bx]).view(np.uint8),
                                      ref.view(np.uint8)), (v, c)
                worst = rc if rc != 0 else worst
            err = np.abs(got.astype(np.float64) - f.astype(np.float64)).max()
            assert err <= tau
        assert st == worst


def test_pipeline_rejects_bad_arguments(B):
    import ctypes as C
    ctx = B.Context()
    dims = (C.c_uint64 * 3)(4, 4, 4)
    ch = (C.c_uint64 * 3)(2, 2, 2)
    total = C.c_uint64(0)
    f = torch.zeros((4, 4, 4), dtype=torch.float32)
    ptrs = (C.c_void_p * 1)(C.c_void_p(f.data_ptr()))
    lib = B.lib()
    assert lib.hpmdr_refactor_pipeline(ctx._p, 0, ptrs, 3, dims, ch, 0, 3, None, C.byref(total),
                                       None, None) == B.ERR_ARG
    assert lib.hpmdr_refactor_pipeline(ctx._p, 1, ptrs, 3, dims, ch, 0, 2, None, C.byref(total),
                                       None, None) == B.ERR_ARG  # 1 or 3 queues
    assert lib.hpmdr_refactor_pipeline(ctx._p, 1, ptrs, 3, dims, ch, 0, 3, None, C.byref(total),
                                       None, None) == 0 and total.value > 0
    small = C.c_uint64(16)
    buf = torch.empty(64, dtype=torch.uint8)
    offs = (C.c_uint64 * 8)()
    sz = (C.c_uint64 * 8)()
    assert lib.hpmdr_refactor_pipeline(ctx._p, 1, ptrs, 3, dims, ch, 0, 3,
                                       C.c_void_p(buf.data_ptr()), C.byref(small), offs,
                                       sz) == B.ERR_ARG
