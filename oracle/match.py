"""Spin-image matching by correlation (test infrastructure only).

Only the tests and bench.py's CPU legs may import this module; it shares no
code with the CUDA library.

Spin images are compared by their linear correlation coefficient, the
similarity measure of spin-image matching (Johnson and Hebert 1999, the
recognition work the paper cites for the algorithm's use): for two images p
and q of N = W*W bins,

    R(p, q) = (N sum p q - sum p sum q) / sqrt((N sum p^2 - (sum p)^2) (N sum q^2 - (sum q)^2)).

Reading: every bin takes part (the matching of that work restricts the sums
to bins where both images hold data; over all bins R is a plain dot product
of centred, unit-length images, a dense contraction); an image with no
variance correlates 0 with everything.  For each scene image the k model
images of highest R are reported, highest first, equal values by smaller
index.
"""
import numpy as np


def unit_centred(images):
    """Rows of (image - its mean) / its centred norm, FP64; zero rows for
    images without variance."""
    x = np.asarray(images, dtype=np.float64).reshape(len(images), -1)
    c = x - x.mean(axis=1, keepdims=True)
    nrm = np.sqrt((c * c).sum(axis=1, keepdims=True))
    return np.divide(c, nrm, out=np.zeros_like(c), where=nrm > 0)


def correlations(scene, model):
    """R of every (scene, model) pair: [n_scene, n_model] FP64."""
    return unit_centred(scene) @ unit_centred(model).T


def best_matches(scene, model, k):
    """(indices [n_scene, k], R [n_scene, k]) of each scene image's k best
    model images, highest R first, ties by smaller index."""
    r = correlations(scene, model)
    order = np.lexsort((np.broadcast_to(np.arange(r.shape[1]), r.shape), -r), axis=1)[:, :k]
    return order.astype(np.int32), np.take_along_axis(r, order, axis=1)
