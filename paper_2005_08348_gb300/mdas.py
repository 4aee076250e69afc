"""Python binding of the C ABI in include/mdas.h (argument marshalling only).

Every computation runs in the CUDA library libmdas.so; this module only
converts numpy arrays to pointers and back.  PyTorch supplies the CUDA stream
and, by default, device memory through its caching allocator.  Importing this
module fails loudly if the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None
_keep_callbacks = []

MDAS_FP32, MDAS_FP64 = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
          4: "unstable state", 5: "timeout", 6: "busy"}
MAX_PAIRS = 64


class MdasError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Desc(C.Structure):
    _fields_ = [
        ("n_beads", C.c_int32), ("n_lipids", C.c_int32), ("beads_per_lipid", C.c_int32),
        ("n_bead_types", C.c_int32), ("n_lipid_types", C.c_int32),
        ("box", C.c_double * 3),
        ("pos", C.c_void_p), ("vel", C.c_void_p),
        ("lipid_first_bead", C.c_void_p), ("lipid_type", C.c_void_p), ("lipid_bead_type", C.c_void_p),
        ("water_bead_type", C.c_int32),
        ("eps", C.c_void_p), ("sigma", C.c_void_p), ("charge", C.c_void_p),
        ("bonds", C.c_void_p), ("n_bonds", C.c_int32),
        ("angles", C.c_void_p), ("n_angles", C.c_int32),
        ("kb", C.c_double), ("b0", C.c_double), ("ktheta", C.c_double), ("theta0_deg", C.c_double),
        ("rc", C.c_double), ("eps_r", C.c_double), ("eps_rf", C.c_double),
        ("temperature", C.c_double), ("dt", C.c_double), ("tau_t", C.c_double), ("mass", C.c_double),
        ("list_skin", C.c_double),
        ("seed", C.c_uint64), ("system_id", C.c_uint32), ("precision", C.c_int32),
        ("cuda_stream", C.c_void_p), ("dev_alloc", _ALLOC), ("dev_free", _FREE), ("alloc_ctx", C.c_void_p),
        ("p_ref", C.c_double), ("tau_p", C.c_double), ("compressibility", C.c_double), ("nstpcouple", C.c_int32),
        ("box_margin", C.c_double),
    ]


class EnergyTerms(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("lj", "rf", "bond", "angle", "kinetic", "potential", "total")] + \
               [("pairs", C.c_int64)]


class SwapStats(C.Structure):
    _fields_ = [("trials", C.c_int64), ("null_trials", C.c_int64), ("accepted", C.c_int64), ("rounds", C.c_int32)]


class MoveResult(C.Structure):
    _fields_ = [("w", C.c_double), ("u", C.c_double), ("accepted", C.c_int32), ("n_pairs", C.c_int32),
                ("pairs", C.c_int32 * (2 * MAX_PAIRS))]


class StateView(C.Structure):
    _fields_ = [("pos_fixed", C.c_void_p), ("pos", C.c_void_p), ("vel", C.c_void_p), ("lipid_type", C.c_void_p),
                ("step", C.c_uint64), ("trial", C.c_uint64), ("move", C.c_uint64), ("at_step", C.c_uint64),
                ("list_ref", C.c_void_p), ("list_valid", C.c_int32), ("ke_valid", C.c_int32),
                ("ke", C.c_double * 2), ("box", C.c_double * 3), ("box_velocity", C.c_double * 3),
                ("list_box", C.c_double * 3)]


class DeviceView(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("vel", C.c_void_p), ("lipid_type", C.c_void_p),
                ("n_beads", C.c_int32), ("n_lipids", C.c_int32), ("precision", C.c_int32),
                ("vel_stride_bytes", C.c_int32), ("box", C.c_double * 3)]


class _DeviceArray:
    """A device array for torch.as_tensor (the CUDA array interface), holding
    the system it belongs to so that the memory outlives the tensor's use."""

    def __init__(self, ptr, shape, typestr, owner):
        self.__cuda_array_interface__ = dict(shape=tuple(shape), typestr=typestr, data=(int(ptr), False),
                                             version=2, strides=None)
        self._owner = owner


class Counters(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("md_steps", "force_evals", "trials", "null_trials", "accepted",
                                         "moves", "moves_accepted", "kernel_launches", "list_builds",
                                         "item_redos")]


TRIAL_DTYPE = np.dtype([("a", np.int32), ("b", np.int32), ("null", np.int32), ("accepted", np.int32),
                        ("dE", np.float64), ("u", np.float64), ("index", np.uint64)])

EXPORTS = ["mdas_create_system", "mdas_destroy_system", "mdas_forces", "mdas_energy", "mdas_md_steps",
           "mdas_swap_trials", "mdas_trial_log", "mdas_alchemical_move", "mdas_delta_energy", "mdas_get_state",
           "mdas_set_state", "mdas_cell_list", "mdas_batch_run", "mdas_philox", "mdas_set_kernel_timing",
           "mdas_pair_kernel_time", "mdas_set_persistent", "mdas_get_counters", "mdas_last_error", "mdas_status_string",
           "mdas_forces_noalloc", "mdas_server_create", "mdas_server_destroy", "mdas_server_submit",
           "mdas_server_run", "mdas_server_results", "mdas_server_clock", "mdas_system_footprint",
           "mdas_tune_list_skin", "mdas_head_rdf", "mdas_mutation_trials", "mdas_set_soft_core",
           "mdas_wait_timeout_probe", "mdas_box", "mdas_alchemical_move_trace", "mdas_interleaflet_move",
           "mdas_device_ptrs", "mdas_server_add_patch", "mdas_server_submit_to", "mdas_server_patch_state",
           "mdas_server_remove_patch", "mdas_tune_batch", "mdas_set_partitioned", "mdas_set_batch_wave",
           "mdas_get_state_packed", "mdas_set_state_packed", "mdas_set_list_lanes", "mdas_set_trial_path"]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libmdas.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libmdas.so not found at {path}")
        L = C.CDLL(path)
        L.mdas_last_error.restype = C.c_char_p
        L.mdas_status_string.restype = C.c_char_p
        L.mdas_destroy_system.restype = None
        for name in EXPORTS:
            getattr(L, name)
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(st, sysptr=None):
    if st != 0:
        msg = lib().mdas_last_error(sysptr).decode()
        raise MdasError(st, msg)


def _torch_allocator():
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC(alloc), _FREE(free)
    _keep_callbacks.append((a, f))
    return a, f


def _current_stream():
    # torch's default stream is the legacy stream (handle 0), on which CUDA
    # graphs cannot be captured; 0 lets the library use its shared stream
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


def make_desc(m, precision=MDAS_FP32, tau_t=None, dt=None, temperature=None, seed=None, system_id=None,
              eps_rf=None, list_skin=0.0):
    """mdas_system_desc of a `synth.Membrane`; returns (desc, arrays kept alive)."""
    k = dict(pos=np.ascontiguousarray(m.pos, np.float64), vel=np.ascontiguousarray(m.vel, np.float64),
             first=np.ascontiguousarray(m.lipid_first_bead, np.int32),
             lt=np.ascontiguousarray(m.lipid_type, np.int32),
             lbt=np.ascontiguousarray(m.lipid_bead_type, np.int32),
             eps=np.ascontiguousarray(m.eps, np.float64), sig=np.ascontiguousarray(m.sigma, np.float64),
             q=np.ascontiguousarray(m.charge, np.float64), bonds=np.ascontiguousarray(m.bonds, np.int32),
             angles=np.ascontiguousarray(m.angles, np.int32))
    d = Desc()
    d.n_beads, d.n_lipids = m.n_beads, m.n_lipids
    d.beads_per_lipid = m.lipid_bead_type.shape[1]
    d.n_bead_types, d.n_lipid_types = m.eps.shape[0], m.lipid_bead_type.shape[0]
    d.box = (C.c_double * 3)(*[float(x) for x in m.box])
    d.pos, d.vel = _p(k["pos"]), _p(k["vel"])
    d.lipid_first_bead, d.lipid_type, d.lipid_bead_type = _p(k["first"]), _p(k["lt"]), _p(k["lbt"])
    d.water_bead_type = int(m.water_bead_type)
    d.eps, d.sigma, d.charge = _p(k["eps"]), _p(k["sig"]), _p(k["q"])
    d.bonds, d.n_bonds = _p(k["bonds"]), int(m.bonds.shape[0])
    d.angles, d.n_angles = _p(k["angles"]), int(m.angles.shape[0])
    d.kb, d.b0, d.ktheta, d.theta0_deg = m.kb, m.b0, m.ktheta, m.theta0_deg
    d.rc, d.eps_r = m.rc, m.eps_r
    d.eps_rf = m.eps_rf if eps_rf is None else eps_rf
    d.temperature = m.temperature if temperature is None else temperature
    d.dt = m.dt if dt is None else dt
    d.tau_t = m.tau_t if tau_t is None else tau_t
    d.mass = m.mass
    d.list_skin = float(list_skin)
    d.seed = int(m.seed if seed is None else seed)
    d.system_id = int(m.system_id if system_id is None else system_id)
    d.precision = precision
    return d, k


def set_pcouple(d, pcouple):
    """The pressure-coupling fields of a description from a dict of p_ref
    (bar), tau_p (ps), compressibility (1/bar), nstpcouple and box_margin
    (None: constant volume)."""
    if pcouple:
        d.p_ref = float(pcouple.get("p_ref", 1.0))
        d.tau_p = float(pcouple.get("tau_p", 12.0))
        d.compressibility = float(pcouple.get("compressibility", 3e-4))
        d.nstpcouple = int(pcouple.get("nstpcouple", 10))
        d.box_margin = float(pcouple.get("box_margin", 0.05))
    return d


class System:
    """One device-resident membrane system built from a `synth.Membrane`."""

    def __init__(self, m, precision="fp32", stream=None, torch_allocator=True, tau_t=None, dt=None,
                 temperature=None, seed=None, system_id=None, eps_rf=None, list_skin=0.0, pcouple=None):
        """pcouple: None (constant volume) or a dict of p_ref (bar), tau_p (ps),
        compressibility (1/bar), nstpcouple, box_margin (see mdas_system_desc)."""
        L = lib()
        self.m = m
        self.n = m.n_beads
        self.n_lipids = m.n_lipids
        self.precision = MDAS_FP64 if precision in ("fp64", MDAS_FP64, "f64") else MDAS_FP32
        d, k = make_desc(m, self.precision, tau_t, dt, temperature, seed, system_id, eps_rf, list_skin)
        set_pcouple(d, pcouple)
        self.stream = _current_stream() if stream is None else int(stream)
        d.cuda_stream = self.stream or None
        if torch_allocator:
            d.dev_alloc, d.dev_free = _torch_allocator()
        self._ptr = C.c_void_p()
        self._desc_arrays = k
        self._desc_fields = dict(d=d)
        _check(L.mdas_create_system(C.byref(d), C.byref(self._ptr)))
        self.kT = 0.0083144626 * d.temperature

    def _desc_for_noalloc(self, stream=None):
        """A copy of the creation descriptor for mdas_forces_noalloc, with the
        system's current box (positions are fractions of it, and pressure
        coupling or set_state may have changed it since creation)."""
        d = Desc()
        C.pointer(d)[0] = self._desc_fields["d"]
        box, _, _ = self.box()
        d.box = (C.c_double * 3)(*[float(x) for x in box])
        d.dev_alloc, d.dev_free = _ALLOC(), _FREE()
        d.cuda_stream = stream
        return d

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "_ptr", None):
            lib().mdas_destroy_system(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        _check(st, self._ptr)

    # -- evaluation -------------------------------------------------------------
    def forces(self):
        F = np.empty((self.n, 3), np.float64)
        self._ck(lib().mdas_forces(self._ptr, _p(F), None))
        return F

    def potential(self):
        u = C.c_double()
        self._ck(lib().mdas_forces(self._ptr, None, C.byref(u)))
        return u.value

    def energy(self):
        t = EnergyTerms()
        self._ck(lib().mdas_energy(self._ptr, C.byref(t)))
        return {k: getattr(t, k) for k, _ in EnergyTerms._fields_}

    def delta_energy(self, lipids, new_types):
        li = np.ascontiguousarray(lipids, np.int32)
        nt = np.ascontiguousarray(new_types, np.int32)
        dE = C.c_double()
        self._ck(lib().mdas_delta_energy(self._ptr, _p(li), _p(nt), int(li.size), C.byref(dE)))
        return dE.value

    # -- sampling -----------------------------------------------------------------
    def md_steps(self, n_steps, swap_every=0):
        self._ck(lib().mdas_md_steps(self._ptr, C.c_int64(n_steps), C.c_int32(swap_every)))

    def swap_trials(self, n, log=True):
        st = SwapStats()
        rec = np.zeros(n, TRIAL_DTYPE) if log else None
        self._ck(lib().mdas_swap_trials(self._ptr, int(n), C.byref(st), _p(rec)))
        return dict(trials=st.trials, null=st.null_trials, accepted=st.accepted, rounds=st.rounds), rec

    def mutation_trials(self, n, mu=None, log=True):
        """Semi-grand mutations (mdas_mutation_trials); mu: per-type chemical
        potentials (kJ/mol) or None."""
        st = SwapStats()
        rec = np.zeros(n, TRIAL_DTYPE) if log else None
        m = None if mu is None else np.ascontiguousarray(mu, np.float64)
        self._ck(lib().mdas_mutation_trials(self._ptr, int(n), _p(m), C.byref(st), _p(rec)))
        return dict(trials=st.trials, null=st.null_trials, accepted=st.accepted), rec

    def trial_log(self, first, n):
        rec = np.zeros(n, TRIAL_DTYPE)
        self._ck(lib().mdas_trial_log(self._ptr, C.c_uint64(first), int(n), _p(rec)))
        return rec

    def alchemical_move(self, n_pairs, n_lambda, md_per_lambda, pairs=None):
        r = MoveResult()
        pin = None
        if pairs is not None:
            pin = np.ascontiguousarray(np.asarray(pairs).reshape(-1), np.int32)
            n_pairs = pin.size // 2
        self._ck(lib().mdas_alchemical_move(self._ptr, int(n_pairs), int(n_lambda), int(md_per_lambda), _p(pin),
                                            C.byref(r)))
        pr = np.array(r.pairs[: 2 * r.n_pairs], np.int32).reshape(-1, 2)
        return dict(w=r.w, u=r.u, accepted=bool(r.accepted), n_pairs=r.n_pairs, pairs=pr)

    def alchemical_move_trace(self, n_pairs, n_lambda, md_per_lambda, pairs=None, positions=True, velocities=True):
        """mdas_alchemical_move_trace: the move plus, per lambda block, the work
        it added, the positions (fixed point) and the velocities after it."""
        r = MoveResult()
        pin = None
        if pairs is not None:
            pin = np.ascontiguousarray(np.asarray(pairs).reshape(-1), np.int32)
            n_pairs = pin.size // 2
        w = np.zeros(int(n_lambda), np.float64)
        pos = np.zeros((int(n_lambda), self.n, 3), np.uint32) if positions else None
        vel = np.zeros((int(n_lambda), self.n, 3), np.float64) if velocities else None
        self._ck(lib().mdas_alchemical_move_trace(self._ptr, int(n_pairs), int(n_lambda), int(md_per_lambda),
                                                  _p(pin), C.byref(r), _p(w), _p(pos), _p(vel)))
        pr = np.array(r.pairs[: 2 * r.n_pairs], np.int32).reshape(-1, 2)
        return dict(w=r.w, u=r.u, accepted=bool(r.accepted), n_pairs=r.n_pairs, pairs=pr, w_blocks=w,
                    pos_blocks=pos, vel_blocks=vel)

    def interleaflet_move(self, n_pairs, n_lambda, md_per_lambda, head_k=1):
        """mdas_interleaflet_move: an alchemical move whose pairs are drawn
        across the two leaflets."""
        r = MoveResult()
        self._ck(lib().mdas_interleaflet_move(self._ptr, int(n_pairs), int(n_lambda), int(md_per_lambda),
                                              int(head_k), C.byref(r)))
        pr = np.array(r.pairs[: 2 * r.n_pairs], np.int32).reshape(-1, 2)
        return dict(w=r.w, u=r.u, accepted=bool(r.accepted), n_pairs=r.n_pairs, pairs=pr)

    # -- state ------------------------------------------------------------------
    def device_views(self):
        """Zero-copy torch tensors over the system's device state
        (mdas_device_ptrs), read-only by contract: pos [n, 4] int32 (x, y, z
        fixed point and the meta word, as raw bits), vel [n, 4] float32 or
        float64, ltype [n_lipids] int32, and the box."""
        import torch
        v = DeviceView()
        self._ck(lib().mdas_device_ptrs(self._ptr, C.byref(v)))
        vt = "<f8" if v.vel_stride_bytes == 32 else "<f4"
        pos = torch.as_tensor(_DeviceArray(v.pos, (v.n_beads, 4), "<i4", self), device="cuda")
        vel = torch.as_tensor(_DeviceArray(v.vel, (v.n_beads, 4), vt, self), device="cuda")
        lt = torch.as_tensor(_DeviceArray(v.lipid_type, (max(v.n_lipids, 0),), "<i4", self), device="cuda")
        return dict(pos=pos, vel=vel, ltype=lt, box=np.array(list(v.box)))

    def get_state(self):
        pu = np.empty((self.n, 3), np.uint32)
        pos = np.empty((self.n, 3), np.float64)
        vel = np.empty((self.n, 3), np.float64)
        lt = np.empty(max(self.n_lipids, 1), np.int32)
        ref = np.empty((self.n, 3), np.uint32)
        v = StateView(_p(pu), _p(pos), _p(vel), _p(lt), 0, 0, 0, 0, _p(ref))
        self._ck(lib().mdas_get_state(self._ptr, C.byref(v)))
        return dict(pos_u=pu, pos=pos, vel=vel, ltype=lt[: self.n_lipids].copy(), step=v.step, trial=v.trial,
                    move=v.move, at_step=v.at_step, list_ref=ref if v.list_valid else None,
                    ke=(v.ke[0], v.ke[1]) if v.ke_valid else None, box=np.array(list(v.box)),
                    box_velocity=np.array(list(v.box_velocity)),
                    list_box=np.array(list(v.list_box)) if v.list_valid else None)

    def box(self):
        """(box [nm], dL/dt [nm/ps], pressure of the last box update [bar])."""
        b, bv, p = (C.c_double * 3)(), (C.c_double * 3)(), (C.c_double * 3)()
        self._ck(lib().mdas_box(self._ptr, b, bv, p))
        return np.array(list(b)), np.array(list(bv)), np.array(list(p))

    def set_state(self, pos_u=None, pos=None, vel=None, ltype=None, step=0, trial=0, move=0, at_step=0,
                  list_ref=None, ke=None, box=None, box_velocity=None, list_box=None):
        """Install a state.  With list_ref and ke as get_state returned them,
        MD continues exactly as it would have from the saved state."""
        a = None if pos_u is None else np.ascontiguousarray(pos_u, np.uint32)
        b = None if pos is None else np.ascontiguousarray(pos, np.float64)
        c = None if vel is None else np.ascontiguousarray(vel, np.float64)
        d = None if ltype is None else np.ascontiguousarray(ltype, np.int32)
        r = None if list_ref is None else np.ascontiguousarray(list_ref, np.uint32)
        if r is not None and r.size != 3 * self.n:
            raise ValueError("list_ref must hold n_beads x 3 fixed-point positions")
        v = StateView(_p(a), _p(b), _p(c), _p(d), step, trial, move, at_step, _p(r), int(r is not None),
                      int(ke is not None))
        if ke is not None:
            v.ke[0], v.ke[1] = float(ke[0]), float(ke[1])
        if box is not None:
            for a in range(3):
                v.box[a] = float(box[a])
                v.box_velocity[a] = 0.0 if box_velocity is None else float(box_velocity[a])
        if list_box is not None:
            for a in range(3):
                v.list_box[a] = float(list_box[a])
        self._ck(lib().mdas_set_state(self._ptr, C.byref(v)))

    def _packed_args(self, pos4, vel4, lipid_type):
        """Host addresses of packed-state arrays (numpy arrays or CPU torch
        tensors, C-contiguous, the sizes mdas_get_state_packed documents)."""
        vbytes = 32 if self.precision == MDAS_FP64 else 16
        out = []
        for a, nbytes in ((pos4, 16 * self.n), (vel4, vbytes * self.n), (lipid_type, 4 * self.n_lipids)):
            if a is None:
                out.append(None)
                continue
            if hasattr(a, "data_ptr"):                  # a torch tensor
                if a.device.type != "cpu" or not a.is_contiguous() or a.numel() * a.element_size() != nbytes:
                    raise ValueError("packed state: a contiguous CPU tensor of %d bytes is needed" % nbytes)
                out.append(C.c_void_p(a.data_ptr()))
            else:
                if not a.flags["C_CONTIGUOUS"] or a.nbytes != nbytes:
                    raise ValueError("packed state: a C-contiguous array of %d bytes is needed" % nbytes)
                out.append(C.c_void_p(a.ctypes.data))
        return out

    def get_state_packed(self, pos4=None, vel4=None, lipid_type=None):
        """The state in the library's layout into host arrays (mdas_get_state_packed):
        pos4 [n, 4] uint32 (x, y, z fixed point, meta word), vel4 [n, 4] float32
        (FP32 systems) or float64, lipid_type [n_lipids] int32.  Pass numpy arrays
        or (pinned) CPU torch tensors to fill; by default numpy arrays are made."""
        if pos4 is None and vel4 is None and lipid_type is None:
            pos4 = np.empty((self.n, 4), np.uint32)
            vel4 = np.empty((self.n, 4), np.float64 if self.precision == MDAS_FP64 else np.float32)
            lipid_type = np.empty(self.n_lipids, np.int32)
        a, b, c = self._packed_args(pos4, vel4, lipid_type)
        self._ck(lib().mdas_get_state_packed(self._ptr, a, b, c))
        return pos4, vel4, lipid_type

    def set_state_packed(self, pos4=None, vel4=None, lipid_type=None):
        """Install a state in the library's layout (mdas_set_state_packed); the
        step, trial and move counters are kept, the pair list is rebuilt."""
        a, b, c = self._packed_args(pos4, vel4, lipid_type)
        self._ck(lib().mdas_set_state_packed(self._ptr, a, b, c))

    def resume(self, state):
        """set_state with everything get_state returned (an exact continuation)."""
        self.set_state(pos_u=state["pos_u"], vel=state["vel"], ltype=state["ltype"], step=state["step"],
                       trial=state["trial"], move=state["move"], at_step=state["at_step"],
                       list_ref=state.get("list_ref"), ke=state.get("ke"), box=state.get("box"),
                       box_velocity=state.get("box_velocity"), list_box=state.get("list_box"))

    def cell_list(self):
        ids = np.empty(self.n, np.int32)
        nc = (C.c_int32 * 3)()
        self._ck(lib().mdas_cell_list(self._ptr, _p(ids), None, nc))
        ncell = tuple(nc)
        start = np.empty(ncell[0] * ncell[1] * ncell[2] + 1, np.int32)
        self._ck(lib().mdas_cell_list(self._ptr, None, _p(start), None))
        return ids, start, ncell

    def head_rdf(self, lipid_type, head_k=1, r_max=3.0, n_bins=60):
        """In-plane head-bead pair counts per leaflet (mdas_head_rdf):
        (counts [2, n_bins] int64, heads per leaflet [2])."""
        counts = np.zeros(2 * int(n_bins), np.int64)
        nh = np.zeros(2, np.int32)
        self._ck(lib().mdas_head_rdf(self._ptr, int(lipid_type), int(head_k), C.c_double(r_max), int(n_bins),
                                     _p(counts), _p(nh)))
        return counts.reshape(2, int(n_bins)), nh

    def counters(self):
        c = Counters()
        self._ck(lib().mdas_get_counters(self._ptr, C.byref(c)))
        return {k: getattr(c, k) for k, _ in Counters._fields_}

    def set_kernel_timing(self, on=True):
        self._ck(lib().mdas_set_kernel_timing(self._ptr, int(bool(on))))

    def set_soft_core(self, delta):
        """Alchemical path: 0 linear, delta > 0 (nm^2) Eq. 4 soft core (mdas_set_soft_core)."""
        self._ck(lib().mdas_set_soft_core(self._ptr, C.c_double(delta)))

    def wait_timeout_probe(self):
        """Let a grid-barrier wait of the MD kernel expire (raises MdasError,
        status "timeout"); the system then needs set_state or resume."""
        self._ck(lib().mdas_wait_timeout_probe(self._ptr))

    def set_list_lanes(self, lanes):
        """List columns (threads) per bead of this system's pair-list step, 2
        or 4 (mdas_set_list_lanes); all systems of a batch must agree."""
        self._ck(lib().mdas_set_list_lanes(self._ptr, int(lanes)))

    def set_trial_path(self, path):
        """How several exchange trials at once run (mdas_set_trial_path): "auto",
        "speculative" (rounds) or "sequential" (from the pair lists)."""
        code = {"auto": 0, "speculative": 1, "sequential": 2}[path] if isinstance(path, str) else int(path)
        self._ck(lib().mdas_set_trial_path(self._ptr, code))

    def set_partitioned(self, on=True):
        """Batches give this system its own share of the persistent kernel's
        groups (mdas_set_partitioned; the default) or run it in lockstep."""
        self._ck(lib().mdas_set_partitioned(self._ptr, int(bool(on))))

    def set_batch_wave(self, max_beads):
        """Batches led by this system run their MD in waves of at most
        max_beads beads (mdas_set_batch_wave; 0: all at once)."""
        self._ck(lib().mdas_set_batch_wave(self._ptr, C.c_int64(int(max_beads))))

    def set_persistent(self, on=True):
        """MD in the persistent kernel (default) or as separate kernel launches."""
        self._ck(lib().mdas_set_persistent(self._ptr, int(bool(on))))

    def pair_kernel_time(self, reset=False):
        ms, n = C.c_double(), C.c_int64()
        self._ck(lib().mdas_pair_kernel_time(self._ptr, C.byref(ms), C.byref(n), int(bool(reset))))
        return ms.value, n.value


def forces_noalloc(system, pos_fixed_ptr, lipid_type_ptr, f_out_ptr, stream=None):
    """mdas_forces_noalloc for the force field of `system` (a System) on
    caller-owned device buffers (integer addresses), e.g. torch tensor
    data_ptr()s.  Raises MdasError with the returned status."""
    d = system._desc_for_noalloc(stream)
    st = lib().mdas_forces_noalloc(C.byref(d), C.c_void_p(pos_fixed_ptr), C.c_void_p(lipid_type_ptr),
                                   C.c_void_p(f_out_ptr))
    if st != 0:
        raise MdasError(st, "forces_noalloc failed")


JOB_SWAPS, JOB_MD, JOB_MDAS = 0, 1, 2


class Job(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32), ("n_pairs", C.c_int32), ("n_lambda", C.c_int32),
                ("md_per_lambda", C.c_int32)]


class JobResult(C.Structure):
    _fields_ = [("job_id", C.c_int64), ("kind", C.c_int32), ("status", C.c_int32), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("md_steps", C.c_int64), ("trials", C.c_int64),
                ("accepted", C.c_int64), ("w", C.c_double), ("move_accepted", C.c_int32),
                ("state_hash", C.c_uint64)]


class Server:
    """The library's request loop (mdas_server_*): continuous batching of
    jobs on device-resident patches, admission by device-memory footprint."""

    def __init__(self, budget_bytes, max_active, md_quantum=25, keep_state_hash=False, stream=None):
        L = lib()
        L.mdas_server_clock.restype = C.c_double
        L.mdas_server_destroy.restype = None
        self._ptr = C.c_void_p()
        _check(L.mdas_server_create(C.c_size_t(int(budget_bytes)), int(max_active), int(md_quantum),
                                    int(bool(keep_state_hash)), C.c_void_p(stream) if stream else None,
                                    C.byref(self._ptr)))

    def submit(self, m, kind, n=0, n_pairs=8, n_lambda=10, md_per_lambda=5, precision=MDAS_FP32):
        d, keep = make_desc(m, precision)
        j = Job(int(kind), int(n), int(n_pairs), int(n_lambda), int(md_per_lambda))
        jid = C.c_int64()
        _check(lib().mdas_server_submit(self._ptr, C.byref(d), C.byref(j), C.byref(jid)))
        return jid.value

    def add_patch(self, m, precision=MDAS_FP32):
        """A device-resident patch (mdas_server_add_patch); returns its id."""
        d, keep = make_desc(m, precision)
        pid = C.c_int64()
        _check(lib().mdas_server_add_patch(self._ptr, C.byref(d), C.byref(pid)))
        return pid.value

    def submit_to(self, patch_id, kind, n=0, n_pairs=8, n_lambda=10, md_per_lambda=5):
        """Queue a job on a resident patch (mdas_server_submit_to)."""
        j = Job(int(kind), int(n), int(n_pairs), int(n_lambda), int(md_per_lambda))
        jid = C.c_int64()
        _check(lib().mdas_server_submit_to(self._ptr, C.c_int64(patch_id), C.byref(j), C.byref(jid)))
        return jid.value

    def patch_state(self, patch_id, n_beads, n_lipids):
        """Positions (fixed point), velocities and lipid types of an idle resident patch."""
        pu = np.empty((n_beads, 3), np.uint32)
        vel = np.empty((n_beads, 3), np.float64)
        lt = np.empty(max(n_lipids, 1), np.int32)
        v = StateView(_p(pu), None, _p(vel), _p(lt))
        _check(lib().mdas_server_patch_state(self._ptr, C.c_int64(patch_id), C.byref(v)))
        return dict(pos_u=pu, vel=vel, ltype=lt[:n_lipids].copy(), step=v.step, trial=v.trial, move=v.move)

    def remove_patch(self, patch_id):
        _check(lib().mdas_server_remove_patch(self._ptr, C.c_int64(patch_id)))

    def run(self, rounds=1):
        a, q = C.c_int32(), C.c_int32()
        _check(lib().mdas_server_run(self._ptr, int(rounds), C.byref(a), C.byref(q)))
        return a.value, q.value

    def results(self, cap=4096):
        out = (JobResult * cap)()
        n = C.c_int32()
        _check(lib().mdas_server_results(self._ptr, out, int(cap), C.byref(n)))
        return [{k: getattr(out[i], k) for k, _ in JobResult._fields_} for i in range(n.value)]

    def clock(self):
        return lib().mdas_server_clock(self._ptr)

    def close(self):
        if getattr(self, "_ptr", None):
            lib().mdas_server_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint(m, precision=MDAS_FP32, pcouple=None):
    """Device bytes a system of this membrane occupies."""
    d, keep = make_desc(m, precision)
    set_pcouple(d, pcouple)
    L = lib()
    L.mdas_system_footprint.restype = C.c_size_t
    return int(L.mdas_system_footprint(C.byref(d)))


def batch_run(systems, md_steps, swap_trials):
    arr = (C.c_void_p * len(systems))(*[s._ptr.value for s in systems])
    _check(lib().mdas_batch_run(arr, len(systems), int(md_steps), int(swap_trials)), systems[0]._ptr)


def tune_list_skin(models, skins=(0.2, 0.25, 0.3, 0.35, 0.4), md_steps=100, swap_trials=0, rounds=3,
                   precision="fp32", stream=None):
    """Time batches of `models` (synth.Membrane list) at each candidate pair-list
    skin (mdas_tune_list_skin); returns (best skin, {skin: us per MD step})."""
    prec = MDAS_FP64 if precision in ("fp64", MDAS_FP64, "f64") else MDAS_FP32
    keep, descs = [], []
    stream = _current_stream() if stream is None else int(stream)
    for m in models:
        d, k = make_desc(m, prec)
        d.cuda_stream = stream or None
        d.dev_alloc, d.dev_free = _torch_allocator()
        keep.append((d, k))
        descs.append(C.pointer(d))
    arr = (C.POINTER(Desc) * len(descs))(*descs)
    cand = np.ascontiguousarray(skins, np.float64)
    us = np.zeros(len(cand), np.float64)
    best = C.c_double()
    _check(lib().mdas_tune_list_skin(arr, len(descs), _p(cand), len(cand), int(md_steps), int(swap_trials),
                                     int(rounds), _p(us), C.byref(best)))
    return best.value, dict(zip(cand.tolist(), us.tolist()))


def tune_batch(models, skins=(0.2, 0.3, 0.4), waves=(0,), lanes=(2, 4), md_steps=100, swap_trials=0, rounds=3,
               precision="fp32", stream=None):
    """Time batches of `models` at every (list skin, layout, wave size, list
    lanes) candidate (mdas_tune_batch); returns (best skin, best layout
    partitioned?, best wave size, best lanes, {(skin, partitioned, wave,
    lanes): us per MD step})."""
    prec = MDAS_FP64 if precision in ("fp64", MDAS_FP64, "f64") else MDAS_FP32
    keep, descs = [], []
    stream = _current_stream() if stream is None else int(stream)
    for m in models:
        d, k = make_desc(m, prec)
        d.cuda_stream = stream or None
        d.dev_alloc, d.dev_free = _torch_allocator()
        keep.append((d, k))
        descs.append(C.pointer(d))
    arr = (C.POINTER(Desc) * len(descs))(*descs)
    cand = np.ascontiguousarray(skins, np.float64)
    wv = np.ascontiguousarray(waves, np.int64)
    ln = np.ascontiguousarray(lanes, np.int32)
    nw, nn = len(wv), len(ln)
    us = np.zeros(2 * len(cand) * nw * nn, np.float64)
    best, part, wave, lane = C.c_double(), C.c_int32(), C.c_int64(), C.c_int32()
    _check(lib().mdas_tune_batch(arr, len(descs), _p(cand), len(cand), _p(wv), nw, _p(ln), nn, int(md_steps),
                                 int(swap_trials), int(rounds), _p(us), C.byref(best), C.byref(part), C.byref(wave),
                                 C.byref(lane)))
    table = {(float(cand[c // (2 * nw * nn)]), bool((c // (nw * nn)) % 2), int(wv[(c // nn) % nw]), int(ln[c % nn])):
             float(us[c]) for c in range(len(us))}
    return best.value, bool(part.value), wave.value, lane.value, table


def philox(k0, k1, c1, c2, c3, n):
    out = np.empty((n, 4), np.uint32)
    _check(lib().mdas_philox(C.c_uint32(k0), C.c_uint32(k1), C.c_uint32(c1), C.c_uint32(c2), C.c_uint32(c3),
                             int(n), _p(out)))
    return out
