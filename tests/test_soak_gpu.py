"""A seeded randomized soak of the map, map-reduce and scan kernels against the
oracle: 1,200 cases with random sizes (log-uniform up to 2^21 elements, plus tiny ones),
random element offsets (misaligned starts), random fixed launch configurations
(vector width, unroll, block) or the tuned default, over eight stock specs.  Maps
and the exact scans are compared element by element, exact reductions bit for
bit, binary32 sums within their bounds."""
import numpy as np
import pytest
import torch

import oracle
from bounds import compensated_sum_bound, plain_sum_bound
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu

POOL = (1 << 21) + 64
A, B = 2.5, -0.75


def _s():
    return torch.cuda.current_stream().cuda_stream


@pytest.fixture(scope="module")
def data():
    x = inputs.uniform_f32(95, 0, POOL, -2.0, 2.0)
    y = inputs.uniform_f32(95, 1, POOL, -2.0, 2.0)
    ln = inputs.lognormal_signed_f32(95, 2, POOL)
    xi = inputs.int_uniform_i32(95, 3, POOL)
    host = dict(x=x, y=y, ln=ln, xi=xi, xb=inputs.to_bf16_values(x), yb=inputs.to_bf16_values(y))
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items() if k not in ("xb", "yb")}
    dev["xb"] = torch.from_numpy(host["xb"]).to(torch.bfloat16).cuda()
    dev["yb"] = torch.from_numpy(host["yb"]).to(torch.bfloat16).cuda()
    return host, dev


def _decode_f32(out):
    return float(out.cpu().numpy().view(np.float32)[0])


def test_random_soak(data):
    host, dev = data
    rng = np.random.default_rng(96)
    specs = ["lin_comb_f32", "lin_comb_bf16", "dot_f32", "sum_f32_comp", "sum_i32_i64",
             "argmin_f32", "cumsum_excl_i32_i64", "cummax_f32"]
    for case in range(1200):
        name = specs[case % len(specs)]
        n = int(rng.integers(0, 40)) if rng.random() < 0.15 else int(2 ** rng.uniform(5, 21))
        off = int(rng.integers(0, 64))
        cfg = {} if rng.random() < 0.3 else dict(
            vec_bytes=int(rng.choice([16, 32])), items_per_thread=int(rng.choice([1, 2, 4])),
            block=int(rng.choice([32, 64, 128, 256, 512])))
        h = stock.create(name, **cfg)
        tag = (case, name, n, off, cfg)
        if name.startswith("lin_comb"):
            bf = name.endswith("bf16")
            xs, ys = (dev["xb"], dev["yb"]) if bf else (dev["x"], dev["y"])
            es = xs.element_size()
            z = torch.full((n + 8,), -1, dtype=xs.dtype, device="cuda")
            pyc.pyc_map_launch(h, n, [xs.data_ptr() + es * off, ys.data_ptr() + es * off,
                                      z.data_ptr() + es * (off % 8)],
                               pyc.pack_scalars(h, [A, B]), _s())
            torch.cuda.synchronize()
            got = z[off % 8: off % 8 + n].float().cpu().numpy()
            hx, hy = (host["xb"], host["yb"]) if bf else (host["x"], host["y"])
            want = oracle.map_lin_comb_f32ops(A, hx[off:off + n], B, hy[off:off + n], out_bf16=bf)
            assert np.array_equal(got, np.asarray(want, np.float32)), tag
            # nothing outside [off % 8, off % 8 + n) was written
            zc = z.float().cpu().numpy()
            assert np.all(zc[: off % 8] == -1) and np.all(zc[off % 8 + n:] == -1), tag
            continue
        if name.startswith("cum"):
            excl = name == "cumsum_excl_i32_i64"
            xs = dev["xi"] if excl else dev["x"]
            ydt = torch.int64 if excl else torch.float32
            y = torch.full((n + 8,), -1, dtype=ydt, device="cuda")
            ey = y.element_size()
            pyc.pyc_scan_launch(h, n, [xs.data_ptr() + 4 * off, y.data_ptr() + ey * (off % 8)],
                                None, _s())
            pyc.pyc_scan_sync(h, _s())
            yc = y.cpu().numpy()
            got = yc[off % 8: off % 8 + n]
            if excl:
                want = oracle.scan_sum_i32_i64(host["xi"][off:off + n], exclusive=True)
            else:
                want = oracle.scan_max_f32(host["x"][off:off + n])
            assert np.array_equal(got, np.asarray(want, got.dtype)), tag
            assert np.all(yc[: off % 8] == -1) and np.all(yc[off % 8 + n:] == -1), tag
            continue
        out = torch.zeros(2, dtype=torch.int64, device="cuda")
        if name == "dot_f32":
            ptrs = [dev["x"].data_ptr() + 4 * off, dev["y"].data_ptr() + 4 * off]
        elif name == "sum_f32_comp":
            ptrs = [dev["ln"].data_ptr() + 4 * off]
        elif name == "sum_i32_i64":
            ptrs = [dev["xi"].data_ptr() + 4 * off]
        else:
            ptrs = [dev["x"].data_ptr() + 4 * off]
        pyc.pyc_reduce_launch(h, n, ptrs, None, out.data_ptr(), _s())
        torch.cuda.synchronize()
        if name == "dot_f32":
            ref, ab = oracle.dot_f32(host["x"][off:off + n], host["y"][off:off + n])
            assert abs(_decode_f32(out) - ref) <= plain_sum_bound(ab), tag
        elif name == "sum_f32_comp":
            seg = host["ln"][off:off + n]
            ex = oracle.exact_sum_f32(seg)
            assert abs(_decode_f32(out) - ex) <= compensated_sum_bound(ex, oracle.sum_f32(seg)[1]), tag
        elif name == "sum_i32_i64":
            assert int(out.cpu()[0]) == oracle.sum_i32_i64(host["xi"][off:off + n]), tag
        else:
            v, idx = pyc.argf32_from_tensor(out.view(1, 2))
            assert (float(v.cpu()[0]), int(idx.cpu()[0])) == oracle.argmin_f32(
                host["x"][off:off + n]), tag


def test_random_segment_tables(data):
    """80 random segment tables (1 to 600 segments, lengths log-uniform up to 2^17
    with empty segments mixed in, misaligned bases, random configurations): dot
    products within their bounds and int32 -> int64 sums and argmins exact per
    segment, each table launched twice (the second a replay of the cached plan)."""
    host, dev = data
    rng = np.random.default_rng(97)
    for case in range(80):
        nseg = int(rng.integers(1, 600))
        lens = np.where(rng.random(nseg) < 0.1, 0,
                        (2 ** rng.uniform(0, 17, nseg)).astype(np.int64)).astype(np.int64)
        total = int(lens.sum())
        if total > POOL - 64:
            lens = (lens * (POOL - 64) // max(total, 1)).astype(np.int64)
            total = int(lens.sum())
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        base = int(rng.integers(0, 64))
        name = ["dot_f32", "sum_i32_i64", "argmin_f32"][case % 3]
        cfg = {} if rng.random() < 0.4 else dict(
            vec_bytes=int(rng.choice([16, 32])), items_per_thread=int(rng.choice([1, 2, 4])),
            block=int(rng.choice([64, 128, 256, 512])))
        h = stock.create(name, **cfg)
        tag = (case, name, nseg, total, base, cfg)
        if name == "dot_f32":
            ptrs = [dev["x"].data_ptr() + 4 * base, dev["y"].data_ptr() + 4 * base]
            out = torch.zeros(nseg, dtype=torch.float32, device="cuda")
        elif name == "sum_i32_i64":
            ptrs = [dev["xi"].data_ptr() + 4 * base]
            out = torch.zeros(nseg, dtype=torch.int64, device="cuda")
        else:
            ptrs = [dev["x"].data_ptr() + 4 * base]
            out = torch.zeros((nseg, 2), dtype=torch.int64, device="cuda")
        for rep in range(2):
            out.zero_()
            pyc.pyc_reduce_batched(h, nseg, off, ptrs, None, out.data_ptr(), _s())
            torch.cuda.synchronize()
            if name == "dot_f32":
                ref, ab = oracle.dot_segments_f32(off, host["x"][base:base + total],
                                                  host["y"][base:base + total])
                got = out.cpu().numpy().astype(np.float64)
                assert np.all(np.abs(got - ref) <= plain_sum_bound(ab)), tag
            elif name == "sum_i32_i64":
                got = out.cpu().numpy()
                for k in range(nseg):
                    a, b = base + off[k], base + off[k + 1]
                    assert got[k] == oracle.sum_i32_i64(host["xi"][a:b]), tag + (k,)
            else:
                v, idx = pyc.argf32_from_tensor(out)
                v, idx = v.cpu().numpy(), idx.cpu().numpy()
                for k in range(nseg):
                    a, b = base + off[k], base + off[k + 1]
                    assert (float(v[k]), int(idx[k])) == oracle.argmin_f32(host["x"][a:b]), \
                        tag + (k,)
