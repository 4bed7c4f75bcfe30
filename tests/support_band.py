"""Support comparison within a band around the thresholds (test helper).

The support of the GPU path must equal the FP64 oracle's except where the
oracle's |u_j| / d (or ||u_g|| / d for a group) lies within `band` of the
threshold at which the penalty's update (Section 2.2) leaves zero: w_j lambda
for the lasso, MCP and SCAD, alpha w_j lambda for the elastic net, c_k lambda
for the group penalties. u = c + d beta - G beta is taken at the oracle's
solution, with the d of the penalty's update.
"""
import numpy as np

import oracle


def support_mismatches(G, c, d, pen, lam, beta_gpu, beta_ref, band=1e-6):
    """(outside, inside): lists of (index, distance to the threshold in units
    of beta) where the two supports differ, outside and inside the band."""
    G = np.asarray(G, dtype=np.float64)
    beta_ref = np.asarray(beta_ref, dtype=np.float64)
    beta_gpu = np.asarray(beta_gpu, dtype=np.float64)
    p = beta_ref.size
    de = oracle.effective_d(d, pen)
    u = c + de * beta_ref - G @ beta_ref
    if pen.kind in ("grp.lasso", "grp.mcp", "grp.scad"):
        members, cg = pen.group_list(p)
        on_g = np.array([np.any(beta_gpu[m] != 0) for m in members])
        on_r = np.array([np.any(beta_ref[m] != 0) for m in members])
        mag = np.array([np.linalg.norm(u[m]) for m in members])
        thr = cg * lam
    else:
        on_g, on_r = beta_gpu != 0, beta_ref != 0
        mag = np.abs(u)
        thr = pen.weights(p) * lam * (pen.alpha if pen.kind == "enet" else 1.0)
    dist = np.abs(mag - thr) / de
    diff = np.flatnonzero(on_g != on_r)
    outside = [(int(j), float(dist[j])) for j in diff if dist[j] > band]
    inside = [(int(j), float(dist[j])) for j in diff if dist[j] <= band]
    return outside, inside
