"""Small hand-built workloads for the oracle pins (plain data, no method code)."""
import dataclasses

import numpy as np

from paper_2311_12818_gb300 import inputs as I


def custom(name, surfaces, light, targets, xD, nD, xL, k, tau, spq=1, hf_desc=None, hf_heights=None,
           scale=3.4641, tau_random=False, pn=None, **params):
    xD = np.atleast_2d(np.asarray(xD, np.float64))
    nD = np.atleast_2d(np.asarray(nD, np.float64))
    if nD.shape[0] == 1 and xD.shape[0] > 1:
        nD = np.tile(nD, (xD.shape[0], 1))
    B = xD.shape[0] * spq
    xL = np.atleast_2d(np.asarray(xL, np.float64))
    if xL.shape[0] == 1 and B > 1:
        xL = np.tile(xL, (B, 1))
    k = np.broadcast_to(np.asarray(k, np.uint8), (B,)).copy()
    tau = np.broadcast_to(np.asarray(tau, np.uint8), (B,)).copy()
    p = dataclasses.replace(I.Params(dedup_eps=1e-4 * scale), **params)
    return I.Workload(name, np.atleast_2d(np.asarray(surfaces, np.float64)),
                      np.zeros((0, 6)) if hf_desc is None else np.atleast_2d(hf_desc),
                      np.zeros(0) if hf_heights is None else np.asarray(hf_heights, np.float64),
                      np.atleast_2d(np.asarray(targets, np.float64)), np.asarray(light, np.float64),
                      xD, nD, np.zeros(xD.shape[0], np.uint32), spq, xL, k, tau, tau_random,
                      np.ones(B) if pn is None else np.asarray(pn, np.float64), 1, 0x1234567,
                      scale, p, (xD.shape[0], 1))


def mirror_plane(xD, xL, point=True, spq=8, **kw):
    surf = I._surface(I.SURF_RECT, I.MAT_MIRROR, 1, 1, (0, 0, 0), 0, (0, 0, 1), -1, (5, 0, 0), (0, 5, 0))
    if point:
        light = I._light(I.LIGHT_POINT, xL)
    else:
        light = I._light(I.LIGHT_RECT, xL, (0, 0, -1), (0.1, 0, 0), (0, 0.1, 0))
    tg = I._target(I.TARGET_RECT, (0, 0, 0), 0, (1.5, 0, 0), (0, 1.5, 0), (0, 0, 1))
    return custom("mirror_plane", surf, light, tg, xD, (0, 0, -1), xL, 1, 0, spq, **kw)


def flat_interface(xD, xL, etaB=1.33, spq=8, refract=True, receiver_normal=(0, 0, 1), **kw):
    surf = I._surface(I.SURF_RECT, I.MAT_DIELECTRIC, 1.0, etaB, (0, 0, 0), 0, (0, 0, 1), -1,
                      (5, 0, 0), (0, 5, 0))
    light = I._light(I.LIGHT_RECT, xL, (0, 0, -1), (0.1, 0, 0), (0, 0.1, 0))
    tg = I._target(I.TARGET_RECT, (0, 0, 0), 0, (1.5, 0, 0), (0, 1.5, 0), (0, 0, 1))
    return custom("flat_interface", surf, light, tg, xD, receiver_normal, xL, 1,
                  1 if refract else 0, spq, **kw)
