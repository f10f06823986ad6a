"""Helpers of the GPU parity tests: oracle-encoded batches, GPU decode through
the C ABI binding, element-wise comparison with the FP64 oracle."""
import numpy as np

import oracle
import siggen

# FP32 inverse transform vs the FP64 oracle: relative L2 error per stream.
FP32_REL_L2 = 1e-5


def product_domain(o: oracle.Domain):
    from paper_2605_01086_gb300 import codec
    return codec.Domain(o.N, o.E, o.B1, o.B2, o.mu, o.alpha1, tuple(o.A), o.lmax, o.code_len.copy())


def oracle_domains():
    return [oracle.trained_domain(i) for i in range(4)]


def encode_workload(wl: siggen.Workload, domains=None, chunk: int = 256):
    """Oracle-encodes a workload chunk by chunk (bounded host memory)."""
    domains = domains or oracle_domains()
    parts = []
    for c0 in range(0, wl.n_streams, chunk):
        sub = wl.subset(np.arange(c0, min(wl.n_streams, c0 + chunk)))
        flat, offs = siggen.signals(sub.domains, sub.seeds, sub.lengths)
        parts.append(oracle.encode_many(flat, offs, sub.lengths, sub.domains, domains))
        del flat
    return concat_batches(parts)


def concat_batches(parts):
    words = np.concatenate([p.words for p in parts]) if parts else np.zeros(0, np.uint64)
    symlen = np.concatenate([p.symlen for p in parts]) if parts else np.zeros(0, np.uint8)
    n_words = np.concatenate([p.n_words for p in parts])
    word_off = np.zeros(len(n_words), np.uint64)
    if len(n_words) > 1:
        word_off[1:] = np.cumsum(n_words[:-1])
    return oracle.EncodedBatch(words, symlen, word_off, n_words, np.concatenate([p.lengths for p in parts]),
                               np.concatenate([p.domain_idx for p in parts]), parts[0].domains)


def segments_of(batch: oracle.EncodedBatch, out_align: int = 4, out_base: int = 0):
    from paper_2605_01086_gb300 import codec
    out_off = codec.packed_out_offsets(batch.lengths, out_align) + np.uint64(out_base)
    return codec.segments_array(batch.word_off, batch.n_words, batch.lengths, out_off, batch.domain_idx)


def make_plan(batch, out_align=4, out_base=0, **opts):
    from paper_2605_01086_gb300 import Plan
    segs = segments_of(batch, out_align, out_base)
    return Plan([product_domain(d) for d in batch.domains], segs, **opts)


def gpu_decode(plan, batch, want_levels=True, scale=None, out_fill=None):
    import torch
    w, s = plan.to_device(batch.words, batch.symlen)
    out = plan.empty_out()
    if out_fill is not None:
        out.fill_(out_fill)
    lv = torch.empty(max(1, plan.info["n_levels_total"]), dtype=torch.uint8, device=plan.device) if want_levels \
        else None
    plan.decode(w, s, out=out, levels=lv, scale=scale)
    torch.cuda.synchronize()
    return w, s, out, lv


def compare_with_oracle(plan, batch, out, lv, idx=None, tol=FP32_REL_L2, domains=None):
    """Levels bit-exact and samples within tol relative L2, stream by stream."""
    n = batch.n_streams
    idx = np.arange(n) if idx is None else np.asarray(idx)
    ob = batch if domains is None else oracle.EncodedBatch(batch.words, batch.symlen, batch.word_off, batch.n_words,
                                                           batch.lengths, batch.domain_idx, domains)
    xs, out_off, olv, lv_off = oracle.decode_many(ob, idx, want_levels=True)
    out_h = out.cpu().numpy()
    lv_h = lv.cpu().numpy() if lv is not None else None
    worst = 0.0
    for j, i in enumerate(idx):
        S = int(batch.lengths[i])
        seg = plan.segments[i]
        g = out_h[int(seg["out_offset"]):int(seg["out_offset"]) + S].astype(np.float64)
        r = xs[int(out_off[j]):int(out_off[j]) + S]
        nr = np.linalg.norm(r)
        err = np.linalg.norm(g - r)
        rel = err / nr if nr > 0 else err
        worst = max(worst, rel)
        assert rel <= tol, f"stream {i}: rel L2 {rel:.3g} > {tol}"
        if lv_h is not None:
            d = batch.domains[batch.domain_idx[i]]
            L = d.windows(S) * d.E
            a = int(plan.level_offsets[i])
            np.testing.assert_array_equal(lv_h[a:a + L], olv[int(lv_off[j]):int(lv_off[j]) + L],
                                          err_msg=f"levels of stream {i}")
    return worst


def crafted_batch(domains, levels_list, lengths, dom_idx):
    """Packs given level arrays with the oracle's Alg. 1 (no signal, no quantizer)."""
    words, symlen, nw = [], [], []
    for X, di in zip(levels_list, dom_idx):
        d = domains[di]
        codes = oracle.canonical_codes(d.code_len, d.lmax)
        w, s = oracle.pack_symlen(X, codes, d.code_len)
        words.append(w)
        symlen.append(s)
        nw.append(w.size)
    nw = np.array(nw, np.uint64)
    off = np.zeros(len(nw), np.uint64)
    if len(nw) > 1:
        off[1:] = np.cumsum(nw[:-1])
    return oracle.EncodedBatch(np.concatenate(words), np.concatenate(symlen), off, nw,
                               np.array(lengths, np.uint64), np.array(dom_idx, np.int32), list(domains))


def near_level_boundary(d: oracle.Domain, x_win, k: int, level: int) -> bool:
    """True if `level` is what the zone quantizer (Eq. 2, Eq. 3) gives for some
    coefficient within the FP64 rounding bound of the oracle's Eq. 1 coefficient
    of bin k of the window x_win, and another level is too: i.e. that coefficient
    sits on a level boundary.  Two FP64 evaluations of the same N-term sum (with
    cosine arguments written in two algebraically equal ways) differ by a few
    ulp per term, so delta = 2 N ulp of (2/N) sum |x| bounds their distance."""
    x_win = np.asarray(x_win, dtype=np.float64)
    c = float(oracle.dct2(x_win, d.N, d.E)[k])
    delta = 2.0 * d.N * 2.0 ** -52 * float(np.abs(x_win).sum()) * 2.0 / d.N
    z = d.zone(k)
    lo, hi = oracle.quantize(d, z, c - delta), oracle.quantize(d, z, c + delta)
    return lo <= level <= hi and lo != hi
