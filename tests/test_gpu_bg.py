"""Parity of the chaotic Blum-Goldwasser kernels (Sec. 9.2) with the oracle:
ciphertext and y element by element for batches with ragged message counts
and lengths, mixed key sizes (w = 3, 4, 5 within one warp), in-place use,
rejected keys, and the full-size 2^20 x 1024 workload on sampled messages plus
the round trip of every message."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import cuda_or_skip
from paper_1112_5239_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _batch(seed, n_msgs, L, n_keys=64, lo=1 << 30, hi=1 << 31):
    b = W.bg_batch(seed, n_msgs, n_keys, lo, hi)
    m = W.bg_messages(seed + 2, n_msgs, L)
    full = np.random.default_rng(seed + 3).integers(0, 256, size=(n_msgs, L), dtype=np.uint8)
    m[::7] = full[::7]  # every 7th message uses whole bytes: bits above w pass through
    return b, m


def _encrypt(torch, ci, b, m, out=None):
    msg = _dev(torch, m, torch.uint8)
    rej = torch.zeros(1, dtype=torch.int32, device="cuda")
    c, y = ci.bg_encrypt(_dev(torch, b["N"], torch.int64), _dev(torch, b["S0"], torch.uint8),
                         _dev(torch, b["r"], torch.int64), msg, out=msg if out == "inplace" else None, rejected=rej)
    torch.cuda.synchronize()
    return c.cpu().numpy(), y.cpu().numpy().view(np.uint64), int(rej.item())


def _decrypt(torch, ci, b, y, c):
    rej = torch.zeros(1, dtype=torch.int32, device="cuda")
    m = ci.bg_decrypt(_dev(torch, b["p"], torch.int64), _dev(torch, b["q"], torch.int64),
                      _dev(torch, b["S0"], torch.uint8), _dev(torch, y.view(np.int64), torch.int64),
                      _dev(torch, c, torch.uint8), rejected=rej)
    torch.cuda.synchronize()
    return m.cpu().numpy(), int(rej.item())


def _oracle_rows(b, m, rows):
    cs, ys = [], []
    for i in rows:
        c, y, _ = oracle.bg_encrypt(int(b["N"][i]), int(b["S0"][i]), int(b["r"][i]), m[i])
        cs.append(c)
        ys.append(y)
    return np.array(cs, dtype=np.uint8).reshape(len(rows), m.shape[1]), np.array(ys, dtype=np.uint64)


def test_encrypt_decrypt_match_oracle():
    torch, ci = cuda_or_skip()
    b, m = _batch(11, 1000, 333)  # 31.25 warps of messages, 10 full tiles + a 13-chunk tail
    c, y, rej = _encrypt(torch, ci, b, m)
    assert rej == 0
    oc, oy = _oracle_rows(b, m, range(1000))
    assert np.array_equal(c, oc)
    assert np.array_equal(y, oy)
    md, rej = _decrypt(torch, ci, b, y, c)
    assert rej == 0 and np.array_equal(md, m)
    for i in (0, 31, 32, 999):
        assert np.array_equal(oracle.bg_decrypt(int(b["p"][i]), int(b["q"][i]), int(b["S0"][i]), int(y[i]), c[i]),
                              m[i])


@pytest.mark.parametrize("n_msgs,L", [(1, 0), (1, 1), (31, 31), (33, 32), (33, 33), (64, 64), (5, 100)])
def test_edge_sizes(n_msgs, L):
    torch, ci = cuda_or_skip()
    b, m = _batch(12 + L, n_msgs, L, n_keys=8)
    c, y, rej = _encrypt(torch, ci, b, m)
    oc, oy = _oracle_rows(b, m, range(n_msgs))
    assert rej == 0 and np.array_equal(c, oc) and np.array_equal(y, oy)
    if L == 0:
        assert [int(v) for v in y] == [pow(int(r), 2, int(N)) for r, N in zip(b["r"], b["N"])]
    md, _ = _decrypt(torch, ci, b, y, c)
    assert np.array_equal(md, m)


def test_mixed_key_sizes_in_one_warp():
    """Rows alternate keys with w = 3 (the paper's 16-bit moduli), 4 and 5,
    and unbalanced factors (p < 2^16, q near 2^31)."""
    torch, ci = cuda_or_skip()
    n, L = 96, 150
    parts = [W.bg_batch(21, n, 16, 128, 256), W.bg_batch(22, n, 16, 1 << 10, 1 << 11), W.bg_batch(23, n, 16)]
    pu, _ = W.bg_keys(24, 16, 1 << 14, 1 << 16)
    b = {k: np.empty_like(parts[0][k]) for k in parts[0]}
    for i in range(n):
        for k in b:
            b[k][i] = parts[i % 3][k][i]
    for i in range(3, n, 8):  # unbalanced keys
        b["p"][i] = pu[i % 16]
        b["N"][i] = b["p"][i] * b["q"][i]
        b["r"][i] = next(v for v in range(12345, 10**9) if math.gcd(v, int(b["N"][i])) == 1)
    ws = {int(math.floor(math.log2(math.floor(math.log2(int(N)))))) for N in b["N"]}
    assert ws == {3, 4, 5}
    m = W.bg_messages(25, n, L, bits=8)
    c, y, rej = _encrypt(torch, ci, b, m)
    oc, oy = _oracle_rows(b, m, range(n))
    assert rej == 0 and np.array_equal(c, oc) and np.array_equal(y, oy)
    md, rej = _decrypt(torch, ci, b, y, c)
    assert rej == 0 and np.array_equal(md, m)


def test_in_place():
    torch, ci = cuda_or_skip()
    b, m = _batch(31, 100, 77, n_keys=8)
    c, y, _ = _encrypt(torch, ci, b, m, out="inplace")
    oc, oy = _oracle_rows(b, m, range(100))
    assert np.array_equal(c, oc) and np.array_equal(y, oy)


def test_rejected_keys():
    torch, ci = cuda_or_skip()
    b, m = _batch(41, 40, 50, n_keys=8)
    N = b["N"].copy()
    N[3], N[4], N[5] = N[3] + 1, 1, (1 << 62) + 1  # even, below 3, above the Montgomery range
    enc = dict(b, N=N)
    c, y, rej = _encrypt(torch, ci, enc, m)
    assert rej == 3
    assert not c[[3, 4, 5]].any() and not y[[3, 4, 5]].any()
    keep = [i for i in range(40) if i not in (3, 4, 5)]
    oc, oy = _oracle_rows(b, m, keep)
    assert np.array_equal(c[keep], oc) and np.array_equal(y[keep], oy)
    p, q = b["p"].copy(), b["q"].copy()
    p[7] = 1009 * 1019          # 3 mod 4 but composite
    p[8] = 1000000009            # prime, but 1 mod 4
    p[9] = q[9]                  # p == q
    p[10] = (1 << 32) + 15       # above 2^32
    dec = dict(b, p=p, q=q)
    md, rej = _decrypt(torch, ci, dec, y, c)
    assert rej == 4  # rows 3-5 keep valid factors: their y = 0 decrypts to garbage but is not rejected
    assert not md[[7, 8, 9, 10]].any()
    ok = [i for i in keep if i not in (7, 8, 9, 10)]
    assert np.array_equal(md[ok], m[ok])


def test_full_size_sampled_and_round_trip():
    """The throughput workload: 2^20 messages x 1024 chunks, keys from a pool
    of 4096 recipients; 256 sampled messages against the oracle, then every
    message decrypted back on the device."""
    torch, ci = cuda_or_skip()
    n, L = W.BG_2E20x1024
    b = W.bg_batch(51, n)
    g = torch.Generator(device="cuda")
    g.manual_seed(52)
    msg = torch.randint(0, 32, (n, L), dtype=torch.uint8, device="cuda", generator=g)
    c, y = ci.bg_encrypt(_dev(torch, b["N"], torch.int64), _dev(torch, b["S0"], torch.uint8),
                         _dev(torch, b["r"], torch.int64), msg)
    rows = np.unique(np.concatenate([[0, 31, 32, n - 33, n - 1],
                                     np.random.default_rng(53).integers(0, n, size=251)]))
    idx = torch.from_numpy(rows).cuda()
    m_s = msg[idx].cpu().numpy()
    sub = {k: v[rows] for k, v in b.items()}
    oc, oy = _oracle_rows(sub, m_s, range(len(rows)))
    assert np.array_equal(c[idx].cpu().numpy(), oc)
    assert np.array_equal(y[idx].cpu().numpy().view(np.uint64), oy)
    md = ci.bg_decrypt(_dev(torch, b["p"], torch.int64), _dev(torch, b["q"], torch.int64),
                       _dev(torch, b["S0"], torch.uint8), y, c)
    assert torch.equal(md, msg)


@pytest.mark.parametrize("L", [96, 160])
def test_aligned_and_unaligned_rows(L):
    """Lengths that are a multiple of 32 chunks take the per-lane 16-byte path
    when both buffers are 16-byte aligned and the staged path when they are
    not (views at a one-byte offset): separate, in-place and unaligned
    encryption, and decryption of each, equal the oracle."""
    torch, ci = cuda_or_skip()
    n = 70
    b, m = _batch(51 + L, n, L, n_keys=8)
    oc, oy = _oracle_rows(b, m, range(n))
    N, S0, r = _dev(torch, b["N"], torch.int64), _dev(torch, b["S0"], torch.uint8), _dev(torch, b["r"], torch.int64)
    m_al = _dev(torch, m, torch.uint8)
    c_al, y_al = ci.bg_encrypt(N, S0, r, m_al)
    m_ip = _dev(torch, m, torch.uint8)
    c_ip, y_ip = ci.bg_encrypt(N, S0, r, m_ip, out=m_ip)
    buf_in = torch.zeros(n * L + 1, dtype=torch.uint8, device="cuda")
    buf_out = torch.zeros(n * L + 1, dtype=torch.uint8, device="cuda")
    m_un, c_un = buf_in[1:].view(n, L), buf_out[1:].view(n, L)
    m_un.copy_(m_al)
    _, y_un = ci.bg_encrypt(N, S0, r, m_un, out=c_un)
    torch.cuda.synchronize()
    for c, y in ((c_al, y_al), (c_ip, y_ip), (c_un, y_un)):
        assert np.array_equal(c.cpu().numpy(), oc)
        assert np.array_equal(y.cpu().numpy().view(np.uint64), oy)
    md, rej = _decrypt(torch, ci, b, oy, oc)
    assert rej == 0 and np.array_equal(md, m)
    buf_dec = torch.zeros(n * L + 1, dtype=torch.uint8, device="cuda")
    d_un = ci.bg_decrypt(_dev(torch, b["p"], torch.int64), _dev(torch, b["q"], torch.int64), S0, y_un, c_un,
                         out=buf_dec[1:].view(n, L))
    torch.cuda.synchronize()
    assert np.array_equal(d_un.cpu().numpy(), m)
