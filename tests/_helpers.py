"""Helpers shared by the GPU tests: run the CUDA path through the C ABI."""
import numpy as np


def gpu_matvec(w, u=None, nrhs=None, storage=0, orth=-1, eta=None, ktype=None, kparam=None,
               kscale=None, a="default", p=None, leaf=None, repeat=1, host=False,
               far_precision=0, near_precision=0):
    """Construct the HTLR operator of workload w on cuda:0 and apply it to u (N x nrhs
    column-major numpy).  Returns (f, info)."""
    import torch
    from paper_2508_05958_gb300 import htlr
    u = w.u(nrhs=nrhs) if u is None else u
    nrhs = u.shape[1] if u.ndim == 2 else 1
    a = w.a() if isinstance(a, str) else a
    H = htlr.htlr_construct(w.ktype if ktype is None else ktype, w.d, w.n,
                            w.leaf if leaf is None else leaf, w.p if p is None else p,
                            w.eta if eta is None else eta,
                            kscale=w.kscale if kscale is None else kscale,
                            kparam=w.kparam if kparam is None else kparam, a=a,
                            storage=storage, orth=orth, far_precision=far_precision,
                            near_precision=near_precision)
    try:
        info = htlr.htlr_info(H)
        if host:
            U = np.asfortranarray(u.reshape(w.N, nrhs))
            F = np.zeros_like(U, order="F")
            htlr.htlr_matvec_host(H, U, F, nrhs)
            outs = [F]
        else:
            ud = torch.from_numpy(np.ascontiguousarray(u.reshape(w.N, nrhs).T)).cuda()
            outs = []
            for _ in range(repeat):
                fd = torch.full_like(ud, float("nan"))
                htlr.htlr_matvec(H, ud, fd, nrhs)
                htlr.htlr_sync(H)
                outs.append(fd.cpu().numpy().T.copy())
    finally:
        htlr.htlr_free(H)
    return (outs if repeat > 1 else outs[0]), info


def rel(a, b):
    a = np.asarray(a).reshape(len(a), -1)
    b = np.asarray(b).reshape(len(b), -1)
    return max(np.linalg.norm(a[:, c] - b[:, c]) / np.linalg.norm(b[:, c]) for c in range(b.shape[1]))
