"""Spatial tree of the guide samples (Sec. 5.6, "Spatial structures") in the
oracle.  TEST INFRASTRUCTURE ONLY: the CUDA library never imports it.

The samples of the last pass live at 6-D positions p = (x_D, x_L).  The tree
is a binary tree over them following the paper's description:
  * a node holding more than T = floor(c sqrt(|S|)) of its own samples is
    split (c = 1, the paper's recommendation); the leaves hold at most T;
  * the split is at the midpoint of the node's box along the axis with the
    largest extent relative to the root box (receiver and light are planes,
    so a fixed x, y, z cycle would cut flat axes);
  * spatial filtering (the paper's footnote): floor(eps k) samples of the
    left child nearest to the split plane are copied into the right child and
    as many of the right child's into the left (k = the node's own samples,
    eps = 0.1); a node's copies are not passed on when it is split in turn
    (the samples far from its children's boxes are discarded);
  * a query descends from the root by the position of (x_D, x_L).
Positions are FP32 values; boxes, midpoints and distances are formed in FP64,
ties broken by sample index, so the tree is a deterministic function of the
positions.  Leaves are numbered in depth-first order, left child first.
"""
from __future__ import annotations

import math

import numpy as np

MAX_DEPTH = 48


class STree:
    def __init__(self, pos, eps=0.1, c=1.0, max_depth=MAX_DEPTH):
        pos = np.asarray(pos, np.float32).astype(np.float64).reshape(-1, 6)
        self.pos, self.eps, self.max_depth = pos, eps, max_depth
        n = pos.shape[0]
        self.T = max(1, int(math.floor(c * math.sqrt(n))))
        lo, hi = (pos.min(axis=0), pos.max(axis=0)) if n else (np.zeros(6), np.zeros(6))
        self.root_ext = hi - lo
        # node arrays: axis (-1 for a leaf), split, left, right (leaf id in left for a leaf)
        self.axis, self.split, self.left, self.right = [], [], [], []
        self.leaf_own, self.leaf_members, self.leaf_box = [], [], []
        self._build(np.arange(n), np.zeros(0, np.int64), lo.copy(), hi.copy(), 0)

    def _node(self):
        self.axis.append(-1)
        self.split.append(0.0)
        self.left.append(-1)
        self.right.append(-1)
        return len(self.axis) - 1

    def _build(self, own, copies, lo, hi, depth):
        i = self._node()
        ext = hi - lo
        rel = np.where(self.root_ext > 0, ext / np.where(self.root_ext > 0, self.root_ext, 1.0), 0.0)
        if own.size <= self.T or depth >= self.max_depth or not np.any(rel > 0):
            self.left[i] = len(self.leaf_own)
            self.leaf_own.append(np.sort(own))
            self.leaf_members.append(np.union1d(own, copies))
            self.leaf_box.append((lo.copy(), hi.copy()))
            return i
        a = int(np.argmax(rel))  # the first axis of largest relative extent
        mid = 0.5 * (lo[a] + hi[a])
        x = self.pos[own, a]
        L, R = own[x < mid], own[x >= mid]
        m = int(math.floor(self.eps * own.size))
        # nearest to the plane first, ties by index (lexsort: last key is primary)
        to_right = L[np.lexsort((L, mid - self.pos[L, a]))][:m]
        to_left = R[np.lexsort((R, self.pos[R, a] - mid))][:m]
        self.axis[i], self.split[i] = a, mid
        hl, lr = hi.copy(), lo.copy()
        hl[a], lr[a] = mid, mid
        self.left[i] = self._build(L, to_left, lo.copy(), hl, depth + 1)
        self.right[i] = self._build(R, to_right, lr, hi.copy(), depth + 1)
        return i

    @property
    def n_leaves(self):
        return len(self.leaf_own)

    def query(self, p):
        """Leaf of each position p [m, 6]."""
        p = np.asarray(p, np.float32).astype(np.float64).reshape(-1, 6)
        out = np.zeros(p.shape[0], np.int64)
        for j in range(p.shape[0]):
            i = 0
            while self.axis[i] >= 0:
                i = self.left[i] if p[j, self.axis[i]] < self.split[i] else self.right[i]
            out[j] = self.left[i]
        return out

    def expand(self, cell, omega, w, k, tau):
        """Records of the leaves: each leaf's members (own samples and copies,
        ascending sample index) with the leaf as their cell, leaves in order."""
        idx = np.concatenate([m for m in self.leaf_members]) if self.n_leaves else np.zeros(0, np.int64)
        leaf = np.concatenate([np.full(m.size, j, np.uint32) for j, m in enumerate(self.leaf_members)]) \
            if self.n_leaves else np.zeros(0, np.uint32)
        return leaf, np.asarray(omega)[idx], np.asarray(w)[idx], np.asarray(k)[idx], np.asarray(tau)[idx]


def positions(wl, chain_index):
    """(x_D, x_L) of the given chains as FP32, [m, 6]."""
    b = np.asarray(chain_index, np.int64)
    return np.concatenate([wl.xD[b // wl.spq], wl.xL[b]], axis=1).astype(np.float32)
