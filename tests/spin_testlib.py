"""Shared helpers of the tests: run the CUDA path through the C ABI and compare
it with the FP64 oracle."""
import numpy as np

import oracle

TOL_L1 = 1e-4  # per-image L1 error / total weight against the FP64 oracle


def gpu_run(points, normals, W, B, cos_s, query_idx=None, m=None, schedule=None, probe=False, stream=None):
    """Generate on cuda:0 through the C ABI.  Returns (images int32 numpy,
    probe dict or None)."""
    import torch

    import paper_1811_00901_gb300 as spin

    dev = torch.device("cuda:0")
    n = points.shape[0]
    if m is None:
        m = n if query_idx is None else len(query_idx)
    tp = torch.from_numpy(np.ascontiguousarray(points, np.float32)).to(dev)
    tn = torch.from_numpy(np.ascontiguousarray(normals, np.float32)).to(dev)
    tq = None if query_idx is None else torch.from_numpy(np.ascontiguousarray(query_idx, np.int32)).to(dev)
    st = stream or torch.cuda.current_stream(dev)
    mesh = spin.si_mesh_create(tp, tn, n, st)
    try:
        out = torch.full((m, W, W), -7, dtype=torch.int32, device=dev)
        sched = schedule or spin.make_schedule("GSS")
        pr = None
        if probe:
            pr = dict(culled=torch.full((m,), -1, dtype=torch.int64, device=dev),
                      cand_hash=torch.zeros((m,), dtype=torch.int32, device=dev),
                      support=torch.full((m,), -1, dtype=torch.int64, device=dev),
                      worker=torch.full((m,), -1, dtype=torch.int32, device=dev),
                      step=torch.full((m,), -1, dtype=torch.int32, device=dev))
            spin.si_generate_probe(mesh, tq, m, W, B, cos_s, sched, out, stream=st, **pr)
        else:
            spin.si_generate(mesh, tq, m, W, B, cos_s, sched, out, st)
        st.synchronize()
        spin.si_get_stats(mesh)
        res = out.cpu().numpy()
        if pr is not None:
            pr = {k: v.cpu().numpy() for k, v in pr.items()}
            pr["cand_hash"] = pr["cand_hash"].view(np.uint32)
        return res, pr
    finally:
        spin.si_mesh_destroy(mesh)


def compare_with_oracle(gpu_imgs, points, normals, W, B, cos_s, query_idx_all, sample, support=None,
                        require_unflagged=False):
    """Compare GPU images (int32, [m, W, W]) at positions `sample` with the
    oracle.  Membership may differ only on boundary-flagged pairs: each flip
    moves at most weight 1, so the L1 allowance is 1e-4 * total + flagged.
    With require_unflagged the sampled images must have no flagged pair at
    all, so the bound is 1e-4 * total alone.  Returns the worst L1 / total
    seen."""
    sample = np.asarray(sample)
    q = sample if query_idx_all is None else np.asarray(query_idx_all)[sample]
    img, sup, flg = oracle.spin_images(points, normals, W, B, cos_s, query_idx=q.astype(np.int32))
    worst = 0.0
    for k, s in enumerate(sample):
        if require_unflagged:
            assert flg[k] == 0, "image %d has %d flagged pairs" % (s, flg[k])
        g = gpu_imgs[s].astype(np.float64) / 65536.0
        tot = img[k].sum()
        l1 = np.abs(g - img[k]).sum()
        allow = TOL_L1 * max(1.0, tot) + flg[k]
        assert l1 <= allow, "image %d: L1 %.4g > allowed %.4g (total %.1f, flagged %d)" % (s, l1, allow, tot, flg[k])
        # the fixed-point total is exactly 65536 x the contributing count
        gsum = int(gpu_imgs[s].astype(np.int64).sum())
        assert gsum % 65536 == 0
        assert abs(gsum // 65536 - int(sup[k])) <= flg[k]
        if support is not None:
            assert gsum == 65536 * int(support[s])
        if flg[k] == 0:
            worst = max(worst, l1 / max(1.0, tot))
    return worst
