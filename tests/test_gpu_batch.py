"""All 572 sectors of the 5x5 J1-J2 torus (every S^z >= 1/2, momentum and little-group
1-D irrep) built with shared one-sublattice tables and applied in one batched launch
with block vectors k = 1, 4, 8 (fp32 / complex fp32).

Pins: every sector's dimension against the character-projection count; three sectors
bit-exact against the oracle's basis; sampled rows against the oracle's matrix-free
rows; every column of every batched product against the single-sector product, and on
four sectors against the oracle's stored matrix."""
import numpy as np
import pytest

import oracle
import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sectors():
    import paper_1804_05028_gb300 as ed
    probs = w.config_square25_sectors()
    bases = ed.build_sectors(probs)
    return probs, bases


def test_every_sector_dimension(sectors):
    probs, bases = sectors
    assert len(bases) == 572
    dims = [B.dim for B in bases]
    assert dims == [oracle.dimension_formula(p) for p in probs]
    assert sum(dims) == sum(oracle.dimension_formula(p) for p in probs)


def _pick(probs, pred):
    return next(i for i, p in enumerate(probs) if pred(p))


def test_three_sectors_bit_exact(sectors):
    probs, bases = sectors
    picks = [
        _pick(probs, lambda p: p.n_up == 17 and p.is_real() and p.n_sym == 200),   # Gamma, C4v
        _pick(probs, lambda p: p.n_up == 18 and not p.is_real()),                  # complex k
        _pick(probs, lambda p: p.n_up == 19 and p.n_sym == 50),                    # a mirror
    ]
    for i in picks:
        s, t = bases[i].export()
        ob, ost = oracle.basis(probs[i])
        assert np.array_equal(s, ob) and np.array_equal(t.astype(np.int32), ost)


def test_sampled_rows_against_oracle(sectors):
    probs, bases = sectors
    rng = np.random.default_rng(3)
    for i in [_pick(probs, lambda p: p.n_up == 13 and p.n_sym == 200 and p.is_real()),
              _pick(probs, lambda p: p.n_up == 14 and not p.is_real())]:
        p, B = probs[i], bases[i]
        s, _ = B.export()
        x = w.state_uniform(s, 5) + (0 if p.is_real() else 1j * w.state_uniform(s, 6))
        dt = torch.float64 if p.is_real() else torch.complex128
        y = B.apply_H(torch.from_numpy(np.asarray(x)).to(dt).cuda()).cpu().numpy()
        rows = np.sort(rng.choice(s.size, 300, replace=False))
        xf = (lambda q: w.state_uniform(q, 5)) if p.is_real() else \
             (lambda q: w.state_uniform(q, 5) + 1j * w.state_uniform(q, 6))
        y_ref = oracle.rows(p, s[rows], xf)
        assert np.abs(y[rows] - y_ref).max() <= 1e-12 * np.abs(y_ref).max()


@pytest.mark.parametrize("k", [1, 4, 8])
def test_batched_matches_single_sector(sectors, k):
    import paper_1804_05028_gb300 as ed
    probs, bases = sectors
    g = torch.Generator(device="cuda").manual_seed(1804)
    xs, ys = [], []
    for p, B in zip(probs, bases):
        dt = torch.float32 if B.is_real else torch.complex64
        xs.append(torch.randn(B.dim * k, dtype=dt, device="cuda", generator=g))
        ys.append(torch.empty_like(xs[-1]))
    bt = ed.Batch(bases, k=k)
    bt.set_vectors(xs, ys)
    for _ in range(2):                       # first call tunes and captures, second replays
        for y in ys:
            y.fill_(float("nan"))
        bt.apply()
        torch.cuda.synchronize()
        for p, B, x, y in zip(probs, bases, xs, ys):
            if B.dim == 0:
                continue
            X, Y = x.view(B.dim, k), y.view(B.dim, k)
            for v in range(k):
                ref = B.apply_H(X[:, v].contiguous())
                assert torch.isfinite(torch.view_as_real(Y[:, v]) if Y.is_complex() else Y[:, v]).all()
                err = (Y[:, v] - ref).abs().max().item()
                assert err <= 2e-6 * max(ref.abs().max().item(), 1.0), (p.name, v, err)
    assert bt.info()["rows_per_item"] in (32, 64, 128, 256)


def test_misaligned_vectors_rejected(sectors):
    """k >= 2 moves a row's k entries with 16-byte accesses: a vector view that starts 4
    bytes into its allocation is refused on the host, before any launch."""
    import paper_1804_05028_gb300 as ed
    probs, bases = sectors
    sub = [B for B in bases if B.dim][:3]
    xs = [torch.zeros(B.dim * 4 + 1, dtype=torch.float32 if B.is_real else torch.complex64,
                      device="cuda") for B in sub]
    ys = [torch.zeros_like(x) for x in xs]
    bt = ed.Batch(sub, k=4)
    with pytest.raises(ed.EdError, match="16-byte aligned"):
        bt.set_vectors([x[1:] for x in xs], [y[1:] for y in ys])
    bt.set_vectors([x[:-1] for x in xs], [y[:-1] for y in ys])   # aligned views pass
    bt.close()
    # k = 8: a gathered row is 32 or 64 bytes, read with 32-byte loads, so x must be
    # 32-byte aligned; a view 16 bytes in passes the 16-byte check and not this one
    x8 = [torch.zeros(B.dim * 8 + 4, dtype=torch.float32 if B.is_real else torch.complex64,
                      device="cuda") for B in sub]
    y8 = [torch.zeros(B.dim * 8, dtype=x.dtype, device="cuda") for x, B in zip(x8, sub)]
    bt = ed.Batch(sub, k=8)
    with pytest.raises(ed.EdError, match="32-byte aligned"):
        bt.set_vectors([x[(4 if B.is_real else 2):][:B.dim * 8] for x, B in zip(x8, sub)], y8)
    bt.set_vectors([x[:B.dim * 8] for x, B in zip(x8, sub)], y8)
    bt.close()


@pytest.mark.parametrize("k", [1, 2, 8])
def test_batched_sublattice_sectors(k):
    """All 16 momentum sectors of the 16-site chain with a two-block split: the batched
    kernel's block-wise search (not the whole-table variant), real and complex sectors,
    against the single-sector product and, for one sector, the oracle's matrix."""
    import paper_1804_05028_gb300 as ed
    probs = [w.chain(16, 2, k=m, n_up=8) for m in range(16)]
    bases = ed.build_sectors(probs)
    g = torch.Generator(device="cuda").manual_seed(7)
    xs = [torch.randn(B.dim * k, dtype=torch.float32 if B.is_real else torch.complex64,
                      device="cuda", generator=g) for B in bases]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    bt = ed.Batch(bases, k=k)
    bt.set_vectors(xs, ys)
    bt.apply()
    torch.cuda.synchronize()
    for p, B, x, y in zip(probs, bases, xs, ys):
        X, Y = x.view(B.dim, k), y.view(B.dim, k)
        for v in range(k):
            ref = B.apply_H(X[:, v].contiguous())
            err = (Y[:, v] - ref).abs().max().item()
            assert err <= 2e-6 * max(ref.abs().max().item(), 1.0), (p.name, v, err)
    H, bs, _ = oracle.hamiltonian(probs[3])
    X = xs[3].view(bases[3].dim, k).cpu().numpy().astype(np.complex128)
    Y = ys[3].view(bases[3].dim, k).cpu().numpy()
    assert np.abs(Y - H @ X).max() <= 2e-6 * np.abs(H @ X).max()
    bt.close()


def test_whole_table_batch_against_oracle(sectors):
    """The whole-table batched kernel (the variant the 572-sector launch runs) against the
    oracle's stored matrix directly, every column of every block width, on four sectors:
    real Gamma with the full C4v little group, a complex momentum, a mirror little group,
    and the largest sector of the set."""
    import paper_1804_05028_gb300 as ed
    probs, bases = sectors
    largest = int(np.argmax([B.dim for B in bases]))
    picks = [
        _pick(probs, lambda p: p.n_up == 14 and p.is_real() and p.n_sym == 200),
        _pick(probs, lambda p: p.n_up == 14 and not p.is_real()),
        _pick(probs, lambda p: p.n_up == 13 and p.n_sym == 50),
        largest,
    ]
    assert len(set(picks)) == 4 and bases[largest].dim > 200000
    refs = {}
    for i in picks:
        refs[i] = oracle.stored_matrix(probs[i])
    for k in (1, 4, 8):
        g = torch.Generator(device="cuda").manual_seed(1804 + k)
        xs = [torch.randn(B.dim * k, dtype=torch.float32 if B.is_real else torch.complex64,
                          device="cuda", generator=g) for B in bases]
        ys = [torch.full_like(x, float("nan")) for x in xs]
        bt = ed.Batch(bases, k=k)
        bt.set_vectors(xs, ys)
        bt.apply()
        torch.cuda.synchronize()
        for i in picks:
            B = bases[i]
            X = xs[i].view(B.dim, k).cpu().numpy()
            Y = ys[i].view(B.dim, k).cpu().numpy()
            for v in range(k):
                xv = X[:, v].astype(np.complex128 if not B.is_real else np.float64)
                ref = refs[i].matvec(xv)
                err = np.abs(Y[:, v] - ref).max()
                assert err <= 2e-6 * np.abs(ref).max(), (probs[i].name, k, v, err)
        bt.close()


def test_set_vectors_between_applies_on_a_stream(sectors):
    """Vectors swapped between two launches queued on a non-blocking stream: the first
    launch still computes with the first vectors (set_vectors waits for it before it
    rewrites the sector table the launch reads)."""
    import paper_1804_05028_gb300 as ed
    probs, bases = sectors
    sub = [B for B in bases if B.dim][:40]
    g = torch.Generator(device="cuda").manual_seed(5)
    mk = lambda: [torch.randn(B.dim, dtype=torch.float32 if B.is_real else torch.complex64,
                              device="cuda", generator=g) for B in sub]
    xa, xb = mk(), mk()
    ya = [torch.full_like(x, float("nan")) for x in xa]
    yb = [torch.full_like(x, float("nan")) for x in xb]
    bt = ed.Batch(sub, k=1)
    bt.set_vectors(xa, ya)
    bt.apply()                     # tunes and captures (synchronous)
    st = torch.cuda.Stream()
    for _ in range(3):
        for y in ya + yb:
            y.fill_(float("nan"))
        torch.cuda.synchronize()
        bt.set_vectors(xa, ya)
        bt.apply(stream=st)
        bt.set_vectors(xb, yb)
        bt.apply(stream=st)
        st.synchronize()
        for B, x1, y1, x2, y2 in zip(sub, xa, ya, xb, yb):
            assert torch.allclose(y1, B.apply_H(x1), rtol=0, atol=2e-6 * max(1.0, y1.abs().max().item()))
            assert torch.allclose(y2, B.apply_H(x2), rtol=0, atol=2e-6 * max(1.0, y2.abs().max().item()))
    bt.close()
