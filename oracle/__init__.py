"""ctypes front end of the FP64 C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The arithmetic lives in oracle.c; this
file only builds it with gcc, marshals numpy arrays and returns results.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

TAG_THERMO, TAG_SWAP, TAG_MDAS_PAIR, TAG_MDAS_ACC, TAG_AT_THERMO = 1, 2, 3, 4, 5
KB = 0.0083144626


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        # no fused multiply-adds: every expression rounds as written, on any host
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False) -> str | None:
    """The same source built with OpenMP (the energy's cell loop split over
    the host cores, per-thread sums added in thread order): for timing the
    CPU baseline on all cores only; None when the compiler has no OpenMP."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(src):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_OMP + f".{os.getpid()}.tmp"
        r = subprocess.run(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fopenmp", "-fPIC",
                            "-shared", "-o", tmp, src, "-lm"], capture_output=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def lib_omp():
    """The OpenMP build (build_omp), loaded; None when it cannot be built."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            path = build_omp()
            if path is None:
                return None
            _lib_omp = C.CDLL(path)
            _lib_omp.or_energy.restype = C.c_double
    return _lib_omp


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.or_energy.restype = C.c_double
            _lib.or_swap_dE.restype = C.c_double
            _lib.or_swap_dE_full.restype = C.c_double
            _lib.or_work_increment.restype = C.c_double
            _lib.or_bussi_alpha.restype = C.c_double
            _lib.or_chi2.restype = C.c_double
            _lib.or_uniform.restype = C.c_double
            _lib.or_mdas_pairs.restype = C.c_int
            _lib.or_interleaflet_pairs.restype = C.c_int
    return _lib


class _Sys(C.Structure):
    _fields_ = [
        ("n_beads", C.c_int), ("n_lipids", C.c_int), ("bpl", C.c_int), ("n_bt", C.c_int), ("n_lt", C.c_int),
        ("box", C.c_double * 3),
        ("lipid_first", C.c_void_p), ("lbt", C.c_void_p), ("water_bt", C.c_int),
        ("eps", C.c_void_p), ("sigma", C.c_void_p), ("charge", C.c_void_p),
        ("bonds", C.c_void_p), ("nb", C.c_int), ("angles", C.c_void_p), ("na", C.c_int),
        ("kb", C.c_double), ("b0", C.c_double), ("ktheta", C.c_double), ("theta0_deg", C.c_double),
        ("rc", C.c_double), ("eps_r", C.c_double), ("eps_rf", C.c_double),
        ("temperature", C.c_double), ("dt", C.c_double), ("tau_t", C.c_double), ("mass", C.c_double),
        ("tc_group", C.c_void_p),
        ("seed", C.c_uint64), ("system_id", C.c_uint32), ("sc_delta", C.c_double),
    ]


class _State(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("vel", C.c_void_p), ("ltype", C.c_void_p),
                ("step", C.c_uint32), ("trial", C.c_uint32), ("move", C.c_uint32), ("at_step", C.c_uint32)]


class _Trial(C.Structure):
    _fields_ = [("a", C.c_int), ("b", C.c_int), ("null_trial", C.c_int), ("accepted", C.c_int),
                ("dE", C.c_double), ("u", C.c_double)]


class _Baro(C.Structure):
    _fields_ = [("p_ref", C.c_double), ("tau_p", C.c_double), ("beta", C.c_double), ("nst", C.c_int),
                ("boxv", C.c_double * 3), ("M", C.c_double * 3), ("P", C.c_double * 3)]


def barostat(p_ref=1.0, tau_p=12.0, beta=3e-4, nst=10):
    """Parrinello-Rahman state (or_baro) at rest."""
    b = _Baro()
    b.p_ref, b.tau_p, b.beta, b.nst = float(p_ref), float(tau_p), float(beta), int(nst)
    return b


def pr_box_update(dt, box, b, P):
    """or_pr_box_update on a copy of box; b (from barostat()) is advanced in place."""
    bx = (C.c_double * 3)(*[float(x) for x in box])
    pp = (C.c_double * 3)(*[float(x) for x in P])
    lib().or_pr_box_update(C.c_double(dt), bx, C.byref(b), pp)
    return np.array(list(bx))


class _Move(C.Structure):
    _fields_ = [("w", C.c_double), ("u", C.c_double), ("accepted", C.c_int), ("n_pairs", C.c_int)]


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


class Oracle:
    """FP64 reference evaluation of one membrane (a `synth.Membrane` or alike)."""

    def __init__(self, m, tau_t=None, dt=None, temperature=None, seed=None, system_id=None,
                 eps_rf=None, kb=None, ktheta=None, soft_core=0.0, threads=False):
        """threads=True: energies and MD steps through the OpenMP build on all
        host cores (timing only; the tests use the single-thread build)."""
        self.m = m
        self._L = lib_omp() if threads else lib()
        if self._L is None:
            raise RuntimeError("the OpenMP build of the oracle is not available on this host")
        n = m.n_beads
        self.n = n
        self._keep = dict(
            lipid_first=_i32(m.lipid_first_bead), lbt=_i32(m.lipid_bead_type).ravel(),
            eps=_f64(m.eps).ravel(), sigma=_f64(m.sigma).ravel(), charge=_f64(m.charge),
            bonds=_i32(m.bonds).ravel(), angles=_i32(m.angles).ravel(),
        )
        grp = np.ones(n, np.int32)
        grp[: m.n_lipids * m.lipid_bead_type.shape[1]] = 0
        self._keep["tc"] = grp
        k = self._keep
        s = _Sys()
        s.n_beads, s.n_lipids, s.bpl = n, m.n_lipids, m.lipid_bead_type.shape[1]
        s.n_bt, s.n_lt = m.eps.shape[0], m.lipid_bead_type.shape[0]
        s.box = (C.c_double * 3)(*[float(x) for x in m.box])
        s.lipid_first, s.lbt, s.water_bt = _p(k["lipid_first"]), _p(k["lbt"]), int(m.water_bead_type)
        s.eps, s.sigma, s.charge = _p(k["eps"]), _p(k["sigma"]), _p(k["charge"])
        s.bonds, s.nb = _p(k["bonds"]), int(m.bonds.shape[0])
        s.angles, s.na = _p(k["angles"]), int(m.angles.shape[0])
        s.kb = m.kb if kb is None else kb
        s.b0, s.theta0_deg = m.b0, m.theta0_deg
        s.ktheta = m.ktheta if ktheta is None else ktheta
        s.rc, s.eps_r = m.rc, m.eps_r
        s.eps_rf = m.eps_rf if eps_rf is None else eps_rf
        s.temperature = m.temperature if temperature is None else temperature
        s.dt = m.dt if dt is None else dt
        s.tau_t = m.tau_t if tau_t is None else tau_t
        s.mass = m.mass
        s.tc_group = _p(grp)
        s.seed = int(m.seed if seed is None else seed)
        s.system_id = int(m.system_id if system_id is None else system_id)
        s.sc_delta = float(soft_core)
        self.s = s
        self.kT = KB * s.temperature

    # -- energies and forces ------------------------------------------------
    def bead_types(self, ltype):
        bt = np.empty(self.n, np.int32)
        lt = _i32(ltype)
        lib().or_bead_types(C.byref(self.s), _p(lt), _p(bt))
        return bt

    def energy(self, pos_u, ltype=None, btA=None, btB=None, lam=0.0, cells=True, forces=True):
        """Returns (terms, F): terms = dict(lj, rf, bond, angle, total, pairs)."""
        pu = _u32(pos_u).reshape(-1)
        if btA is None:
            btA = self.bead_types(self.m.lipid_type if ltype is None else ltype)
        btA = _i32(btA)
        btB = btA if btB is None else _i32(btB)
        t = np.zeros(6)
        F = np.zeros((self.n, 3)) if forces else None
        self._L.or_energy(C.byref(self.s), _p(pu), _p(btA), _p(btB), C.c_double(lam), int(cells), _p(t),
                          _p(F) if forces else None)
        terms = dict(lj=t[0], rf=t[1], bond=t[2], angle=t[3], total=t[4], pairs=int(t[5]))
        return terms, F

    @property
    def box(self):
        return np.array(list(self.s.box))

    @box.setter
    def box(self, b):
        self.s.box = (C.c_double * 3)(*[float(x) for x in b])

    def pressure(self, pos_u, vel, ltype=None, cells=True):
        """(P [bar], K, Xi [kJ/mol]) diagonals (or_pressure)."""
        pu = _u32(pos_u).reshape(-1)
        v = _f64(vel).reshape(-1)
        bt = self.bead_types(self.m.lipid_type if ltype is None else ltype)
        P, K, X = np.zeros(3), np.zeros(3), np.zeros(3)
        lib().or_pressure(C.byref(self.s), _p(pu), _p(v), _p(bt), int(cells), _p(P), _p(K), _p(X))
        return P, K, X

    def cell_dims(self):
        nc = (C.c_int * 3)()
        lib().or_cell_dims(C.byref(self.s), nc)
        return tuple(nc)

    def cell_list(self, pos_u):
        nc = self.cell_dims()
        ncell = nc[0] * nc[1] * nc[2]
        cell_of = np.empty(self.n, np.int32)
        srt = np.empty(self.n, np.int32)
        start = np.empty(ncell + 1, np.int32)
        pu = _u32(pos_u).reshape(-1)
        lib().or_cell_list(self.n, _p(pu), (C.c_int * 3)(*nc), _p(cell_of), _p(srt), _p(start))
        return cell_of, srt, start

    # -- swaps ----------------------------------------------------------------
    def swap_dE(self, pos_u, ltype, a, b):
        return lib().or_swap_dE(C.byref(self.s), _p(_u32(pos_u).reshape(-1)), _p(_i32(ltype)), int(a), int(b))

    def swap_dE_full(self, pos_u, ltype, a, b, cells=False):
        return lib().or_swap_dE_full(C.byref(self.s), _p(_u32(pos_u).reshape(-1)), _p(_i32(ltype)),
                                     int(a), int(b), int(cells))

    def work_increment(self, pos_u, btA, btB, l0, l1):
        """U_{l1}(x) - U_{l0}(x) over the pairs with a bead whose A and B types
        differ (or_work_increment): the work of one lambda step (Eq. 2)."""
        return lib().or_work_increment(C.byref(self.s), _p(_u32(pos_u).reshape(-1)), _p(_i32(btA)), _p(_i32(btB)),
                                       C.c_double(l0), C.c_double(l1))

    def swap_proposal(self, t):
        a, b, u = C.c_int(), C.c_int(), C.c_double()
        lib().or_swap_proposal(C.byref(self.s), C.c_uint32(t), C.byref(a), C.byref(b), C.byref(u))
        return a.value, b.value, u.value

    def swap_trials(self, pos_u, ltype, t0, n):
        """Sequential trials t0..t0+n-1; returns (new ltype, records)."""
        lt = _i32(ltype).copy()
        recs = (_Trial * max(n, 1))()
        lib().or_swap_trials(C.byref(self.s), _p(_u32(pos_u).reshape(-1)), _p(lt), C.c_uint32(t0), int(n), recs)
        return lt, [dict(a=r.a, b=r.b, null=bool(r.null_trial), accepted=bool(r.accepted), dE=r.dE, u=r.u)
                    for r in recs[:n]]

    def mutation_trials(self, pos_u, ltype, t0, n, mu=None):
        """Semi-grand mutations in order (or_mutation_trials): returns the
        records and the final lipid types."""
        lt = np.array(ltype, np.int32)
        m = np.zeros(16) if mu is None else np.ascontiguousarray(np.pad(np.asarray(mu, np.float64), (0, 16 - len(mu))))
        out = (_Trial * n)()
        lib().or_mutation_trials(C.byref(self.s), _p(_u32(pos_u).reshape(-1)), _p(lt), C.c_uint32(t0), int(n),
                                 _p(m), out)
        recs = [dict(a=r.a, b=r.b, null=r.null_trial, accepted=r.accepted, dE=r.dE, u=r.u) for r in out]
        return recs, lt

    # -- dynamics -------------------------------------------------------------
    def state(self, pos_u=None, vel=None, ltype=None, step=0, trial=0, move=0, at_step=0):
        m = self.m
        return dict(pos_u=_u32(m.pos_u if pos_u is None else pos_u).reshape(self.n, 3).copy(),
                    vel=_f64(m.vel if vel is None else vel).reshape(self.n, 3).copy(),
                    ltype=_i32(m.lipid_type if ltype is None else ltype).copy(),
                    step=step, trial=trial, move=move, at_step=at_step)

    def _cstate(self, st):
        cs = _State()
        cs.pos, cs.vel, cs.ltype = _p(st["pos_u"]), _p(st["vel"]), _p(st["ltype"])
        cs.step, cs.trial, cs.move, cs.at_step = st["step"], st["trial"], st["move"], st["at_step"]
        return cs

    def _back(self, st, cs):
        st["step"], st["trial"], st["move"], st["at_step"] = cs.step, cs.trial, cs.move, cs.at_step

    def md_steps(self, st, n_steps, swap_every=0, cells=True):
        """Advance st in place; returns the trial records."""
        cs = self._cstate(st)
        nt = n_steps // swap_every if swap_every > 0 else 0
        recs = (_Trial * max(nt, 1))()
        self._L.or_md_steps(C.byref(self.s), C.byref(cs), int(n_steps), int(swap_every), int(cells), recs)
        self._back(st, cs)
        return [dict(a=r.a, b=r.b, null=bool(r.null_trial), accepted=bool(r.accepted), dE=r.dE, u=r.u)
                for r in recs[:nt]]

    def md_steps_npt(self, st, baro, n_steps, swap_every=0, cells=True):
        """Constant-pressure MD (or_md_steps_npt): st, baro and self.box advance."""
        cs = self._cstate(st)
        nt = n_steps // swap_every if swap_every > 0 else 0
        recs = (_Trial * max(nt, 1))()
        lib().or_md_steps_npt(C.byref(self.s), C.byref(cs), C.byref(baro), int(n_steps), int(swap_every),
                              int(cells), recs)
        self._back(st, cs)
        return [dict(a=r.a, b=r.b, null=bool(r.null_trial), accepted=bool(r.accepted), dE=r.dE, u=r.u)
                for r in recs[:nt]]

    def mdas_pairs(self, ltype, move, n_pairs, max_tries=None):
        pairs = np.zeros(2 * n_pairs, np.int32)
        mt = 64 * n_pairs + 64 if max_tries is None else max_tries
        np_ = lib().or_mdas_pairs(C.byref(self.s), _p(_i32(ltype)), C.c_uint32(move), int(n_pairs), int(mt), _p(pairs))
        return pairs[: 2 * np_].reshape(-1, 2)

    def leaflets(self, pos_u, head_k=1):
        """Leaflet of every lipid (or_leaflets): 0 when bead head_k lies above the last bead."""
        leaf = np.empty(max(self.s.n_lipids, 1), np.int32)
        lib().or_leaflets(C.byref(self.s), _p(_u32(pos_u).reshape(-1)), int(head_k), _p(leaf))
        return leaf[: self.s.n_lipids]

    def interleaflet_pairs(self, pos_u, ltype, move, n_pairs, head_k=1, max_tries=None):
        """Pairs of an exchange between the leaflets for move `move` (or_interleaflet_pairs)."""
        pairs = np.zeros(2 * max(n_pairs, 1), np.int32)
        mt = 64 * n_pairs + 64 if max_tries is None else max_tries
        np_ = lib().or_interleaflet_pairs(C.byref(self.s), _p(_u32(pos_u).reshape(-1)), _p(_i32(ltype)),
                                          C.c_uint32(move), int(n_pairs), int(mt), int(head_k), _p(pairs))
        return pairs[: 2 * np_].reshape(-1, 2)

    def mdas_move(self, st, n_pairs, n_lambda, md_per_lambda, pairs=None, cells=True):
        cs = self._cstate(st)
        res = _Move()
        pin = None
        if pairs is not None:
            pin = _i32(np.asarray(pairs).reshape(-1))
            n_pairs = pin.size // 2
        pout = np.zeros(2 * max(n_pairs, 1), np.int32)
        lib().or_mdas_move(C.byref(self.s), C.byref(cs), int(n_pairs), int(n_lambda), int(md_per_lambda),
                           _p(pin) if pin is not None else None, int(cells), _p(pout), C.byref(res))
        self._back(st, cs)
        return dict(w=res.w, u=res.u, accepted=bool(res.accepted), n_pairs=res.n_pairs,
                    pairs=pout[: 2 * res.n_pairs].reshape(-1, 2).copy())

    # -- random numbers -------------------------------------------------------
    def head_rdf(self, pos_u, ltype, lipid_type, head_k=1, r_max=3.0, n_bins=60):
        """Pair counts [2, n_bins] of the in-plane head-bead distribution per
        leaflet and the heads per leaflet [2] (or_head_rdf)."""
        counts = np.zeros(2 * n_bins, np.int64)
        nh = np.zeros(2, np.int32)
        pu = _u32(pos_u).reshape(-1)
        lt = _i32(ltype)
        lib().or_head_rdf(C.byref(self.s), _p(pu), _p(lt), int(lipid_type), int(head_k), C.c_double(r_max),
                          int(n_bins), _p(counts), _p(nh))
        return counts.reshape(2, n_bins), nh

    def bussi_alpha(self, K, nf, kt, i0, i1, tag=TAG_THERMO):
        return lib().or_bussi_alpha(C.byref(self.s), C.c_double(K), int(nf), C.c_double(kt),
                                    C.c_uint32(i0), C.c_uint32(i1), C.c_uint32(tag))

    def chi2(self, k, i0, i1, tag=TAG_THERMO):
        return lib().or_chi2(C.byref(self.s), C.c_uint32(i0), C.c_uint32(i1), C.c_uint32(tag), int(k))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    out = (C.c_uint32 * 4)()
    lib().or_philox(c, k, out)
    return [int(x) for x in out]


def uniform53(a, b):
    return lib().or_uniform(C.c_uint32(a), C.c_uint32(b))
