"""Float64 reference of the image-quality metrics (Sec. III-F, Model Evaluation).

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU leg may
import it; the library never does).  Plain numpy, one formula per function, from
the definitions the paper gives or cites:

- MAE (Sec. III-F, the equation for the mean absolute error): mean over the image
  points of |c_est - c_true|, with c_est = 1 / (bicubic slowness at the point).
- Coherence factor (Mallart and Fink, cited in Sec. III-F), here over receive
  subapertures: with S_j(p) = sum_i B_ij(p) the image of receive block j,
  CF(p) = |sum_j S_j|^2 / (n_sub sum_j |S_j|^2).
- Lag-one coherence (Long et al., cited), over receive subapertures and a region:
  LOC = mean over j of  Re sum_p S_j conj(S_{j+1}) / sqrt(sum_p |S_j|^2 sum_p |S_{j+1}|^2).
- Common-midpoint correlation coefficient (Simson et al., cited): the mean over
  patches and common-midpoint pairs (i,j)~(i+1,j-1), j != i+1, of
  rho = |sum_p B_ij conj(B_{i+1,j-1})| / sqrt(sum_p |B_ij|^2 sum_p |B_{i+1,j-1}|^2).
- Contrast (dB) = 20 log10(mean_in / mean_out) of the envelope |sum_ij B_ij|;
  CNR = |mean_in - mean_out| / sqrt(var_in + var_out);
  generalized CNR (Rodriguez-Molares et al., cited) = 1 - sum_b min(h_in(b), h_out(b))
  with h the normalised histograms of the envelope over nbins equal bins spanning
  [min, max] of the envelope over both regions.
Regions: roi[p] = 1 inside the target, 2 background, 0 not used.  CF is averaged
and LOC formed over the background region.
"""
import numpy as np


def receive_images(B, nsub):
    """S[j][p] = sum_i B_ij(p), B indexed [i * nsub + j][p]."""
    return np.asarray(B).reshape(nsub, nsub, -1).sum(axis=0)


def coherence_factor(S):
    num = np.abs(S.sum(axis=0)) ** 2
    den = S.shape[0] * (np.abs(S) ** 2).sum(axis=0)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)


def lag_one_coherence(S, sel):
    S = S[:, sel]
    vals = []
    for j in range(S.shape[0] - 1):
        e1 = (np.abs(S[j]) ** 2).sum()
        e2 = (np.abs(S[j + 1]) ** 2).sum()
        if e1 > 0 and e2 > 0:
            vals.append(np.real((S[j] * np.conj(S[j + 1])).sum()) / np.sqrt(e1 * e2))
        else:
            vals.append(0.0)
    return float(np.mean(vals)) if vals else 0.0


def cm_pairs(nsub):
    return [(i, j) for i in range(nsub - 1) for j in range(1, nsub) if j != i + 1]


def cmcc(B, nsub, n_patch, patch_npix):
    B = np.asarray(B).reshape(nsub * nsub, n_patch, patch_npix)
    rhos = []
    for (i, j) in cm_pairs(nsub):
        a = B[i * nsub + j]
        b = B[(i + 1) * nsub + (j - 1)]
        z = (a * np.conj(b)).sum(axis=1)
        den = np.sqrt((np.abs(a) ** 2).sum(axis=1) * (np.abs(b) ** 2).sum(axis=1))
        rhos.append(np.where(den > 0, np.abs(z) / np.where(den > 0, den, 1.0), 0.0))
    return float(np.mean(rhos)) if rhos else 0.0


def contrast_cnr_gcnr(env, roi, nbins=256):
    env = np.asarray(env, np.float64)
    a, b = env[roi == 1], env[roi == 2]
    mi, mo = a.mean(), b.mean()
    contrast = 20.0 * np.log10(mi / mo)
    cnr = abs(mi - mo) / np.sqrt(a.var() + b.var())
    both = np.concatenate([a, b])
    lo, hi = both.min(), both.max()
    span = hi - lo if hi > lo else 1.0
    ia = np.minimum(((a - lo) / span * nbins).astype(np.int64), nbins - 1)
    ib = np.minimum(((b - lo) / span * nbins).astype(np.int64), nbins - 1)
    ha = np.bincount(ia, minlength=nbins) / a.size
    hb = np.bincount(ib, minlength=nbins) / b.size
    gcnr = 1.0 - np.minimum(ha, hb).sum()
    return float(contrast), float(cnr), float(gcnr), float(mi), float(mo)


def speed_mae(c_est, c_true):
    return float(np.mean(np.abs(np.asarray(c_est, np.float64) - np.asarray(c_true, np.float64))))


def image_metrics(B, nsub, n_patch, patch_npix, roi, nbins=256):
    """The metric set of one forward pass: dict of CF, LOC, CMCC, contrast, CNR, gCNR."""
    roi = np.asarray(roi)
    S = receive_images(B, nsub)
    env = np.abs(np.asarray(B).sum(axis=0))
    cf = coherence_factor(S)
    bg = roi == 2
    contrast, cnr, gcnr, mi, mo = contrast_cnr_gcnr(env, roi, nbins)
    return dict(cf_mean=float(cf[bg].mean()), loc=lag_one_coherence(S, bg),
                cmcc=cmcc(B, nsub, n_patch, patch_npix), contrast_db=contrast, cnr=cnr,
                gcnr=gcnr, mean_in=mi, mean_out=mo)
