"""The warm-up block's reading and what it costs, on the weighted-cascade
2^20-vertex workload (k = 50, eps = 0.5).

Algorithm 1 builds the codebook from the first block of sets, but IMM does not
know theta when sampling starts.  The reading used here is W = ceil(T_1 / 8),
T_1 being IMM's first sampling target.  A vertex that no warm-up set holds gets
no code, so its occurrences in later Huffman sets go to the copy arrays.  The
test recomputes that share with the oracle:
- for this reading;
- for the first eighth of the final pool, which would need theta before sampling;
- for the whole pool, where by construction nothing is left uncoded.
"""
import numpy as np

import oracle
import synth


def test_warmup_reading_and_its_uncoded_share():
    w = synth.WORKLOADS["wc_rmat1m"]
    g = w.graph()
    op = oracle.Pool(g, oracle.IC, w.rr_seed)
    r = op.imm(w.k, w.eps, w.ell)
    theta, T1 = int(r["theta"]), int(r["round_T"][0])
    assert theta == 45579 and (T1 + 7) // 8 == 695
    off, verts = op.concat(0, theta)
    sizes = np.diff(off.astype(np.int64))
    in_huffman_set = np.repeat(32 * sizes <= g.n, sizes)  # the per-set density cut (reading 13)

    def uncoded_share(W):
        f = op.warmup_freq(W, 32)
        return float(((f[verts] == 0) & in_huffman_set).sum()) / len(verts)

    assert abs(uncoded_share((T1 + 7) // 8) - 0.6776) < 5e-4   # this reading
    assert abs(uncoded_share(theta // 8) - 0.3242) < 5e-4      # first eighth of the final pool
    assert uncoded_share(theta) == 0.0                          # every set in the warm-up block
