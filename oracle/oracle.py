"""CPU oracle for the 2-D volume potential of arXiv 2205.04401 (FP64).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` call this; the library never does.  It
shares no code with the CUDA path: its quadrature tables come from
``oracle/gen_rules.py`` and its arithmetic from ``oracle/oracle.c``.

Steps, in the paper's order (Section 3.6, "subtract-and-add"):
  1. nodes y_j and weights W_j of every triangle (Theorem 3.1, affine map);
  2. far sum over all nodes as point charges W_j f_j (Section 3.6);
  3. S(x) by point location (Appendix A.5) and N(x) by the Bernstein-ellipse
     test (Section 4.1, Eqs. rho0 / threeE);
  4. per (x, T) in N(x) u S(x): subtract the far-rule contribution of T's
     nodes and add the near (Section 3.3) or self (Section 3.4) integral.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(HERE, "oracle.c")
_BUILD = os.path.join(HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
NB = 15
MAXQ = 1024


class OrParams(C.Structure):
    _fields_ = [
        ("nq", C.c_int), ("far_degree", C.c_int),
        ("fx", C.c_double * MAXQ), ("fy", C.c_double * MAXQ), ("fw", C.c_double * MAXQ),
        ("far_what", C.c_double), ("far_cn", C.c_double),
        ("nn", C.c_int), ("near_degree", C.c_int),
        ("nx", C.c_double * MAXQ), ("ny", C.c_double * MAXQ), ("nw", C.c_double * MAXQ),
        ("near_what", C.c_double), ("near_cn", C.c_double),
        ("ng", C.c_int), ("gr", C.c_double * 16), ("gw", C.c_double * 16),
        ("nl", C.c_int), ("lx", C.c_double * 32), ("lw", C.c_double * 32),
        ("bidx_a", C.c_int * NB), ("bidx_b", C.c_int * NB), ("Linv", (C.c_double * NB) * NB),
        ("eps", C.c_double), ("depth_cap", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (no FMA contraction)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
    return _lib


def load_tables(path=None):
    path = path or os.path.join(HERE, "rules_oracle.json")
    with open(path) as fh:
        raw = json.load(fh)
    hx = lambda a: np.array([float.fromhex(v) for v in a])
    out = {}
    for k, v in raw.items():
        if k == "basis":
            out[k] = dict(index=v["index"], Linv=np.array([[float.fromhex(x) for x in row] for row in v["Linv"]]))
            continue
        d = {}
        for kk, vv in v.items():
            if isinstance(vv, list):
                d[kk] = hx(vv)
            elif isinstance(vv, str):
                d[kk] = float.fromhex(vv)
            else:
                d[kk] = vv
        out[k] = d
    return out


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


D = C.c_double
I32 = C.c_int32
I64 = C.c_int64
U8 = C.c_uint8


class Oracle:
    """FP64 reference evaluator for one far rule: 'far16', 'far19', or a rule
    dict (x, y, w, degree, what) such as gen_rules.conical_rule(n)."""

    def __init__(self, rule="far19", eps: float = 1e-12, far_cn: float = 1.0, near_cn: float = 12.0,
                 depth_cap: int = 30, nl: int = 16, tables=None):
        t = tables or load_tables()
        self.tables = t
        fr = t[rule] if isinstance(rule, str) else {k: (np.asarray(v, np.float64) if isinstance(v, list) else v)
                                                    for k, v in rule.items()}
        nr, gg = t["near33"], t["ggq8"]
        gl = t["gl16"] if nl == 16 else t["gl7"]
        p = OrParams()
        p.nq = len(fr["w"])
        p.far_degree = int(fr["degree"])
        for i in range(p.nq):
            p.fx[i], p.fy[i], p.fw[i] = fr["x"][i], fr["y"][i], fr["w"][i]
        p.far_what, p.far_cn = fr["what"], far_cn
        p.nn = len(nr["w"])
        p.near_degree = int(nr["degree"])
        for i in range(p.nn):
            p.nx[i], p.ny[i], p.nw[i] = nr["x"][i], nr["y"][i], nr["w"][i]
        p.near_what, p.near_cn = nr["what"], near_cn
        p.ng = len(gg["r"])
        for i in range(p.ng):
            p.gr[i], p.gw[i] = gg["r"][i], gg["w"][i]
        p.nl = len(gl["x"])
        for i in range(p.nl):
            p.lx[i], p.lw[i] = gl["x"][i], gl["w"][i]
        idx = t["basis"]["index"]
        for i in range(NB):
            p.bidx_a[i], p.bidx_b[i] = idx[i][0], idx[i][1]
            for j in range(NB):
                p.Linv[i][j] = t["basis"]["Linv"][i][j]
        p.eps = eps
        p.depth_cap = depth_cap
        self.p = p
        self.nq = p.nq
        self.rule = rule
        self.L = lib()

    # -- step 1
    def nodes(self, vxy, tri):
        vxy = np.ascontiguousarray(vxy, np.float64)
        tri = np.ascontiguousarray(tri, np.int32)
        nt = len(tri)
        tri_ccw = np.empty_like(tri)
        yxy = np.empty((nt * self.nq, 2))
        W = np.empty(nt * self.nq)
        J = np.empty(nt)
        rc = self.L.or_nodes(_ptr(vxy, D), I64(len(vxy)), _ptr(tri, I32), I64(nt), C.byref(self.p),
                             _ptr(tri_ccw, I32), _ptr(yxy, D), _ptr(W, D), _ptr(J, D))
        if rc != 0:
            raise ValueError(f"or_nodes failed: {rc}")
        return tri_ccw, yxy, W, J

    # -- step 3a
    def locate(self, vxy, tri_ccw, pts):
        pts = np.ascontiguousarray(pts, np.float64)
        out = np.empty(len(pts), np.int32)
        self.L.or_locate(_ptr(vxy, D), _ptr(tri_ccw, I32), I64(len(tri_ccw)), _ptr(pts, D), I64(len(pts)),
                         _ptr(out, I32))
        return out

    # -- step 2
    def far(self, yxy, W, f, txy, tnode):
        f = np.ascontiguousarray(np.atleast_2d(f), np.float64)
        txy = np.ascontiguousarray(txy, np.float64)
        tnode = np.ascontiguousarray(tnode, np.int64)
        d, N = f.shape
        out = np.empty((d, len(txy)))
        self.L.or_far(_ptr(yxy, D), _ptr(W, D), I64(N), _ptr(f, D), C.c_int(d), _ptr(txy, D), _ptr(tnode, I64),
                      I64(len(txy)), _ptr(out, D))
        return out

    # -- step 3b
    def lists(self, vxy, tri_ccw, J, txy, tself):
        txy = np.ascontiguousarray(txy, np.float64)
        tself = np.ascontiguousarray(tself, np.int32)
        m = len(txy)
        cnt = np.empty(m, np.int64)
        self.L.or_lists(_ptr(vxy, D), _ptr(tri_ccw, I32), _ptr(J, D), I64(len(tri_ccw)), C.byref(self.p),
                        _ptr(txy, D), _ptr(tself, I32), I64(m), _ptr(cnt, I64), None, None, None)
        row = np.zeros(m + 1, np.int64)
        np.cumsum(cnt, out=row[1:])
        otri = np.empty(row[-1], np.int32)
        okind = np.empty(row[-1], np.uint8)
        self.L.or_lists(_ptr(vxy, D), _ptr(tri_ccw, I32), _ptr(J, D), I64(len(tri_ccw)), C.byref(self.p),
                        _ptr(txy, D), _ptr(tself, I32), I64(m), _ptr(cnt, I64), _ptr(row, I64), _ptr(otri, I32),
                        _ptr(okind, U8))
        return row, otri, okind

    def near_pred(self, vxy, tri_ccw, J, pts, tids):
        pts = np.ascontiguousarray(pts, np.float64)
        tids = np.ascontiguousarray(tids, np.int64)
        out = np.empty(len(pts), np.uint8)
        self.L.or_near_pred(_ptr(vxy, D), _ptr(tri_ccw, I32), _ptr(J, D), C.byref(self.p), _ptr(pts, D),
                            _ptr(tids, I64), I64(len(pts)), _ptr(out, U8))
        return out.astype(bool)

    # -- step 4
    def weights(self, vxy, tri_ccw, J, txy, pt, ptri, pkind, pown):
        pt = np.ascontiguousarray(pt, np.int64)
        ptri = np.ascontiguousarray(ptri, np.int32)
        pkind = np.ascontiguousarray(pkind, np.uint8)
        pown = np.ascontiguousarray(pown, np.int32)
        n = len(pt)
        out = np.empty((n, self.nq))
        stats = np.empty(n, np.int64)
        capped = I64(0)
        self.L.or_weights(_ptr(vxy, D), _ptr(tri_ccw, I32), _ptr(J, D), C.byref(self.p), _ptr(txy, D),
                          _ptr(pt, I64), _ptr(ptri, I32), _ptr(pkind, U8), _ptr(pown, I32), I64(n),
                          _ptr(out, D), _ptr(stats, I64), C.byref(capped))
        return out, stats, int(capped.value)

    def pair_moments(self, A, B, Cv, J, x, kind):
        m = np.empty(NB)
        st = I64(0)
        A = np.ascontiguousarray(A, np.float64)
        B = np.ascontiguousarray(B, np.float64)
        Cv = np.ascontiguousarray(Cv, np.float64)
        self.L.or_pair_moments(C.byref(self.p), _ptr(A, D), _ptr(B, D), _ptr(Cv, D), D(J), D(x[0]), D(x[1]),
                               C.c_int(kind), _ptr(m, D), C.byref(st))
        return m, int(st.value)

    def basis(self, xi, eta):
        xi = np.ascontiguousarray(xi, np.float64)
        eta = np.ascontiguousarray(eta, np.float64)
        out = np.empty((len(xi), NB))
        self.L.or_basis(C.byref(self.p), _ptr(xi, D), _ptr(eta, D), I64(len(xi)), _ptr(out, D))
        return out

    def self_panel_counts(self, A, B, Cv, x):
        out = np.empty(6, np.int32)
        A = np.ascontiguousarray(A, np.float64)
        B = np.ascontiguousarray(B, np.float64)
        Cv = np.ascontiguousarray(Cv, np.float64)
        self.L.or_self_panel_counts(_ptr(A, D), _ptr(B, D), _ptr(Cv, D), D(x[0]), D(x[1]), _ptr(out, I32))
        return out

    # -- curved elements (blending map; see oracle.c)
    @staticmethod
    def _curves(curves, nt):
        cidx = np.ascontiguousarray(curves["cidx"], np.int32)
        coef = np.ascontiguousarray(curves["coef"], np.float64)
        assert len(cidx) == nt and coef.ndim == 3 and coef.shape[1] == 2
        return cidx, coef, int(coef.shape[2] - 1)

    def nodes_curved(self, vxy, tri, curves):
        vxy = np.ascontiguousarray(vxy, np.float64)
        tri = np.ascontiguousarray(tri, np.int32)
        nt = len(tri)
        cidx, coef, K = self._curves(curves, nt)
        tri_ccw = np.empty_like(tri)
        yxy = np.empty((nt * self.nq, 2))
        W = np.empty(nt * self.nq)
        J = np.empty(nt)
        rc = self.L.or_nodes_curved(_ptr(vxy, D), I64(len(vxy)), _ptr(tri, I32), I64(nt), _ptr(cidx, I32),
                                    _ptr(coef, D), C.c_int(K), C.byref(self.p), _ptr(tri_ccw, I32), _ptr(yxy, D),
                                    _ptr(W, D), _ptr(J, D))
        if rc != 0:
            raise ValueError(f"or_nodes_curved failed: {rc}")
        return tri_ccw, yxy, W, J

    def locate_curved(self, vxy, tri_ccw, curves, pts):
        cidx, coef, K = self._curves(curves, len(tri_ccw))
        pts = np.ascontiguousarray(pts, np.float64)
        out = np.empty(len(pts), np.int32)
        self.L.or_locate_curved(_ptr(vxy, D), _ptr(tri_ccw, I32), I64(len(tri_ccw)), _ptr(cidx, I32), _ptr(coef, D),
                                C.c_int(K), _ptr(pts, D), I64(len(pts)), _ptr(out, I32))
        return out

    def map_curved(self, vxy, tri_ccw, curves, T, xi, eta):
        cidx, coef, K = self._curves(curves, len(tri_ccw))
        T = np.ascontiguousarray(T, np.int64)
        xi = np.ascontiguousarray(xi, np.float64)
        eta = np.ascontiguousarray(eta, np.float64)
        y = np.empty((len(T), 2))
        det = np.empty(len(T))
        self.L.or_map_curved(_ptr(np.ascontiguousarray(vxy, np.float64), D), _ptr(tri_ccw, I32), _ptr(cidx, I32),
                             _ptr(coef, D), C.c_int(K), _ptr(T, I64), _ptr(xi, D), _ptr(eta, D), I64(len(T)),
                             _ptr(y, D), _ptr(det, D))
        return y, det

    def inverse_curved(self, vxy, tri_ccw, curves, T, pts):
        cidx, coef, K = self._curves(curves, len(tri_ccw))
        T = np.ascontiguousarray(T, np.int64)
        pts = np.ascontiguousarray(pts, np.float64)
        ref = np.empty((len(T), 2))
        it = np.empty(len(T), np.int32)
        self.L.or_inverse_curved(_ptr(np.ascontiguousarray(vxy, np.float64), D), _ptr(tri_ccw, I32),
                                 _ptr(cidx, I32), _ptr(coef, D), C.c_int(K), _ptr(T, I64), _ptr(pts, D),
                                 I64(len(T)), _ptr(ref, D), _ptr(it, I32))
        return ref, it

    def weights_curved(self, s, pt, ptri, pkind, pown):
        cidx, coef, K = self._curves(s["curves"], len(s["tri"]))
        pt = np.ascontiguousarray(pt, np.int64)
        ptri = np.ascontiguousarray(ptri, np.int32)
        pkind = np.ascontiguousarray(pkind, np.uint8)
        pown = np.ascontiguousarray(pown, np.int32)
        n = len(pt)
        out = np.empty((n, self.nq))
        stats = np.empty(n, np.int64)
        capped = I64(0)
        self.L.or_weights_curved(_ptr(s["vxy"], D), _ptr(s["tri"], I32), _ptr(s["J"], D), _ptr(cidx, I32),
                                 _ptr(coef, D), C.c_int(K), C.byref(self.p), _ptr(s["yxy"], D), _ptr(s["W"], D),
                                 _ptr(s["txy"], D), _ptr(pt, I64), _ptr(ptri, I32), _ptr(pkind, U8),
                                 _ptr(pown, I32), I64(n), _ptr(out, D), _ptr(stats, I64), C.byref(capped))
        return out, stats, int(capped.value)

    def pair_moments_curved(self, s, T, x, kind):
        cidx, coef, K = self._curves(s["curves"], len(s["tri"]))
        m = np.empty(NB)
        st = I64(0)
        self.L.or_pair_moments_curved(C.byref(self.p), _ptr(s["vxy"], D), _ptr(s["tri"], I32), _ptr(s["J"], D),
                                      _ptr(cidx, I32), _ptr(coef, D), C.c_int(K), I64(T), D(x[0]), D(x[1]),
                                      C.c_int(kind), _ptr(m, D), C.byref(st))
        return m, int(st.value)

    # -- composition
    def setup(self, vxy, tri, node_targets=True, extra=None, curves=None):
        """Nodes, targets, S(x) and lists.  Targets: all nodes (if
        node_targets), then the extra points.  curves: optional curved
        elements {"cidx": [nt], "coef": [ncurve][2][K+1]}."""
        vxy = np.ascontiguousarray(vxy, np.float64)
        if curves is not None:
            tri_ccw, yxy, W, J = self.nodes_curved(vxy, tri, curves)
        else:
            tri_ccw, yxy, W, J = self.nodes(vxy, tri)
        N = len(W)
        parts, tnode, tself = [], [], []
        if node_targets:
            parts.append(yxy)
            tnode.append(np.arange(N, dtype=np.int64))
            tself.append((np.arange(N) // self.nq).astype(np.int32))
        if extra is not None and len(extra):
            extra = np.ascontiguousarray(extra, np.float64)
            parts.append(extra)
            tnode.append(np.full(len(extra), -1, np.int64))
            tself.append(self.locate_curved(vxy, tri_ccw, curves, extra) if curves is not None
                         else self.locate(vxy, tri_ccw, extra))
        txy = np.ascontiguousarray(np.vstack(parts))
        return dict(vxy=vxy, tri=tri_ccw, yxy=yxy, W=W, J=J, txy=txy, tnode=np.concatenate(tnode),
                    tself=np.concatenate(tself), N=N, curves=curves)

    def own_index(self, s, t_idx, ptri):
        tn = s["tnode"][t_idx]
        own = np.where((tn >= 0) & (tn // self.nq == ptri), tn - ptri.astype(np.int64) * self.nq, -1)
        return own.astype(np.int32)

    def potential(self, s, f, targets=None):
        """u at the selected targets (all by default) for densities f ([d][N]
        node values).  Returns (u [d][m], info)."""
        f = np.ascontiguousarray(np.atleast_2d(f), np.float64)
        idx = np.arange(len(s["txy"])) if targets is None else np.asarray(targets, np.int64)
        txy = s["txy"][idx]
        ufar = self.far(s["yxy"], s["W"], f, txy, s["tnode"][idx])
        row, ptri, pkind = self.lists(s["vxy"], s["tri"], s["J"], txy, s["tself"][idx])
        pt_local = np.repeat(np.arange(len(idx)), np.diff(row))
        pt = idx[pt_local]
        pown = self.own_index(s, pt, ptri)
        if s.get("curves") is not None:
            Cw, stats, capped = self.weights_curved(s, pt, ptri, pkind, pown)
        else:
            Cw, stats, capped = self.weights(s["vxy"], s["tri"], s["J"], s["txy"], pt, ptri, pkind, pown)
        fT = f.reshape(f.shape[0], -1, self.nq)           # [d][T][nq]
        corr = np.einsum("pk,dpk->dp", Cw, fT[:, ptri, :])
        u = ufar.copy()
        for k in range(f.shape[0]):
            u[k] += np.bincount(pt_local, weights=corr[k], minlength=len(idx))
        info = dict(row=row, ptri=ptri, pkind=pkind, C=Cw, stats=stats, capped=capped, ufar=ufar)
        return u, info
