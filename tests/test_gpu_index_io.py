"""dade_save_index / dade_load_index round trip (GPU only).

A loaded index must be the saved one: every exported field equal, the same
search results bit for bit (FP32 path and low-precision prefilter), and a
damaged file must be refused before it can reach a kernel.
"""
import os

import numpy as np
import pytest

from paper_2411_17229_gb300 import dade, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17229_gb300 import build
    build.build()
    base, queries, _ = synth.make("c1_gauss_10k_d128", n=5000, nq=64)
    ix = dade.Index(torch.from_numpy(base).cuda(), 40, kmeans_iters=3, seed=7, eps_pairs=3000,
                    lead_format=dade.LEAD_FP8, lead_dims=32, tail_from=48)
    return ix, torch.from_numpy(queries).cuda()


def _search(ix, q, flags):
    ids = torch.empty(q.shape[0], 10, dtype=torch.int64, device="cuda")
    d = torch.empty(q.shape[0], 10, dtype=torch.float32, device="cuda")
    ix.query(q, 10, 6, 0.1, 32, ids, d, flags=flags)
    ix.sync()
    return ids.cpu().numpy(), d.cpu().numpy()


def test_round_trip(built, tmp_path):
    ix, q = built
    path = str(tmp_path / "c1.dade")
    ix.save(path)
    back = dade.Index.load(path)
    for f in ("n", "d", "d_pad", "n_clusters", "max_list", "eps_kept", "data_bytes", "kmeans_iters",
              "lead_format", "lead_dims", "tail_from"):
        assert getattr(back.info, f) == getattr(ix.info, f), f
    for field in range(11):
        a, b = ix.export(field), back.export(field)
        assert a.dtype == b.dtype and np.array_equal(a, b), field
    for flags in (0, dade.FLAG_LEAD, dade.FLAG_ROW_TAIL, dade.FLAG_LEAD | dade.FLAG_ROW_TAIL):
        i0, d0 = _search(ix, q, flags)
        i1, d1 = _search(back, q, flags)
        assert np.array_equal(i0, i1) and np.array_equal(d0.view(np.uint32), d1.view(np.uint32))


def test_damaged_files_refused(built, tmp_path):
    ix, _ = built
    path = str(tmp_path / "ok.dade")
    ix.save(path)
    raw = bytearray(open(path, "rb").read())
    info = ix.info
    d, n, nc, nb = info.d, info.n, info.n_clusters, info.d_pad // 16
    # header (88 B), then (u64 size, bytes) sections: mean, basis, eigenvalues, prefix sums, rho, assign, lists
    off = 88
    for size in (8 * d, 8 * d * d, 8 * d, 8 * (d + 1), 8 * (nb - 1) * info.eps_kept, 4 * n):
        assert int.from_bytes(raw[off:off + 8], "little") == size
        off += 8 + size
    assert int.from_bytes(raw[off:off + 8], "little") == 24 * nc
    first = off + 8                                     # ListMeta {i64 base, i64 slot, i32 len, i32 np}
    np_ = int.from_bytes(raw[first + 20:first + 24], "little")
    cases = {
        "len_beyond_padding": (first + 16, (np_ + 4).to_bytes(4, "little")),
        "base_beyond_data": (first, (1 << 40).to_bytes(8, "little")),
        "magic": (0, b"XXXX"),
    }
    for name, (pos, patch) in cases.items():
        bad = bytearray(raw)
        bad[pos:pos + len(patch)] = patch
        p = str(tmp_path / f"{name}.dade")
        open(p, "wb").write(bytes(bad))
        with pytest.raises(dade.DadeError) as e:
            dade.Index.load(p)
        assert e.value.status == dade.EINVAL, name
    p = str(tmp_path / "short.dade")
    open(p, "wb").write(bytes(raw[: len(raw) // 2]))
    with pytest.raises(dade.DadeError) as e:
        dade.Index.load(p)
    assert e.value.status == dade.EIO
    with pytest.raises(dade.DadeError) as e:
        dade.Index.load(os.path.join(str(tmp_path), "missing.dade"))
    assert e.value.status == dade.EIO
