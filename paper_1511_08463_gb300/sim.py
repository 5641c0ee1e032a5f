"""Thin Python wrapper over the C ABI: builds the C descriptors from a ``workloads.Workload``,
owns the device workspace (a torch uint8 tensor) and marshals calls.  No solver arithmetic here."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import binding as B

_EDGE = {"left": 0, "right": 1, "bottom": 2, "top": 3}
_COMP = {"ux": 0, "uy": 1, "alpha": 2}


def mesh_desc(w) -> B.pf_mesh_desc:
    d = B.pf_mesh_desc()
    d.kind = B.PF_MESH_CROSSED if w.kind == "crossed" else B.PF_MESH_RIGHT
    d.nx, d.ny = w.nx, w.ny
    d.x0, d.y0, d.lx, d.ly = w.x0, w.y0, w.lx, w.ly
    for edge, comps in w.fixed.items():
        for comp, g in comps.items():
            d.fixed[_EDGE[edge]][_COMP[comp]] = 1
            d.load[_EDGE[edge]][_COMP[comp]] = g
    if len(w.pins) > B.PF_MAX_PINS or len(w.alpha_boxes) > B.PF_MAX_BOXES:
        raise ValueError("too many pins or boxes")
    d.n_pins = len(w.pins)
    for k, (x2, y2, comp, g) in enumerate(w.pins):
        d.pin_x2[k], d.pin_y2[k], d.pin_comp[k], d.pin_load[k] = x2, y2, _COMP[comp], g
    d.n_boxes = len(w.alpha_boxes)
    for k, (xl, xh, yl, yh, v) in enumerate(w.alpha_boxes):
        d.box[k][0], d.box[k][1], d.box[k][2], d.box[k][3] = xl, xh, yl, yh
        d.box_value[k] = v
    if w.mode_I is not None:
        d.mode_I = 1
        m = w.mode_I
        d.mode_I_param[0], d.mode_I_param[1] = m["KI"], m["x_tip0"]
        d.mode_I_param[2], d.mode_I_param[3] = m["v"], m["y_line"]
    return d


def material(w) -> B.pf_material:
    m = B.pf_material()
    m.E, m.nu, m.Gc, m.ell, m.k_ell = w.E, w.nu, w.Gc, w.ell, w.k_ell
    m.model = B.PF_AT1 if w.model == "AT1" else B.PF_AT2
    m.plane = B.PF_PLANE_STRAIN if w.plane == "strain" else B.PF_PLANE_STRESS
    m.beta, m.pen = w.beta, w.pen
    return m


def make_opts(**kw) -> B.pf_solver_opts:
    o = B.pf_solver_opts()
    B.check(B.load().pf_default_opts(C.byref(o)))
    names = {"AM": B.PF_ALGO_AM, "ORAM": B.PF_ALGO_ORAM, "ORAM_N": B.PF_ALGO_ORAM_N,
             "fp64": B.PF_FP64, "mixed": B.PF_MIXED}
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, names.get(v, v) if isinstance(v, str) else v)
    return o


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream


class Context:
    def __init__(self, device: int = 0):
        self.lib = B.load()
        self.device = device
        h = C.c_void_p()
        B.check(self.lib.pf_ctx_create(device, C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            self.lib.pf_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sim:
    """One resident fracture simulation (state u, alpha, alpha_prev in device memory)."""

    def __init__(self, w, ctx: Context | None = None):
        self.lib = B.load()
        self.ctx = ctx or Context(0)
        self.w = w
        self.desc = mesh_desc(w)
        nbytes = self.lib.pf_workspace_bytes(C.byref(self.desc), B.PF_FP64)
        if nbytes == 0:
            raise B.PFError(B.PF_EINVAL, self.lib.pf_last_error().decode())
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8,
                                     device=f"cuda:{self.ctx.device}")
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        h = C.c_void_p()
        B.check(self.lib.pf_create_mesh(self.ctx.h, C.byref(self.desc), C.c_void_p(aligned),
                                        nbytes, C.byref(h)))
        self.h = h
        self.mat = material(w)
        B.check(self.lib.pf_set_material(self.h, C.byref(self.mat)))
        nn, ne, lv = C.c_int64(), C.c_int64(), C.c_int32()
        B.check(self.lib.pf_sim_info(self.h, C.byref(nn), C.byref(ne), C.byref(lv)))
        self.n_nodes, self.n_elements, self.levels = nn.value, ne.value, lv.value
        self.workspace_bytes = nbytes

    def close(self):
        if getattr(self, "h", None):
            self.lib.pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- main entry points ----------------------------------------------------------------
    def load_step(self, t: float, dT: float = 0.0, opts=None, stream=None, allow_notconv=False):
        o = opts or make_opts(omega=self.w.omega)
        L = B.pf_load(t, dT)
        rep = B.pf_step_report()
        st = self.lib.pf_load_step(self.h, C.byref(L), C.byref(o), C.c_void_p(_stream(stream)),
                                   C.byref(rep))
        B.check(st, (B.PF_OK, B.PF_ENOTCONV) if allow_notconv else (B.PF_OK,))
        return rep.as_dict()

    def energy(self, stream=None):
        out = (C.c_double * 3)()
        B.check(self.lib.pf_energy(self.h, C.c_void_p(_stream(stream)), out))
        return list(out)

    def get_fields(self):
        n = self.n_nodes
        u = np.empty((n, 2))
        a = np.empty(n)
        ap = np.empty(n)
        B.check(self.lib.pf_get_fields(self.h, u.ctypes.data, a.ctypes.data, ap.ctypes.data))
        return u, a, ap

    def set_fields(self, u=None, alpha=None, alpha_prev=None):
        def p(x, shape):
            if x is None:
                return None, None
            arr = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(shape))
            return arr, arr.ctypes.data

        ua, up = p(u, (self.n_nodes, 2))
        aa, ap_ = p(alpha, (self.n_nodes,))
        pa, pp = p(alpha_prev, (self.n_nodes,))
        B.check(self.lib.pf_set_fields(self.h, up, ap_, pp))

    def autotune(self, opts=None, stream=None) -> dict:
        o = opts or make_opts(omega=self.w.omega)
        r = B.pf_tune_report()
        B.check(self.lib.pf_autotune(self.h, C.byref(o), C.c_void_p(_stream(stream)), C.byref(r)))
        return r.as_dict()

    def set_load(self, t: float, dT: float = 0.0):
        L = B.pf_load(t, dT)
        B.check(self.lib.pf_set_load(self.h, C.byref(L)))

    # ---- operator entry points ------------------------------------------------------------
    def elastic_apply(self, x: torch.Tensor, masked: bool = False, stream=None) -> torch.Tensor:
        prec = B.PF_FP64 if x.dtype == torch.float64 else B.PF_MIXED
        x = x.contiguous()
        y = torch.empty_like(x)
        B.check(self.lib.pf_op_elastic_apply(self.h, prec, int(masked), _ptr(x), _ptr(y),
                                             C.c_void_p(_stream(stream))))
        return y

    def elastic_residual(self, stream=None, precision="fp64"):
        r = torch.empty(2 * self.n_nodes, dtype=torch.float64, device=self.workspace.device)
        n2 = C.c_double()
        prec = B.PF_MIXED if precision == "mixed" else B.PF_FP64
        B.check(self.lib.pf_op_elastic_residual(self.h, prec, _ptr(r), C.byref(n2),
                                                C.c_void_p(_stream(stream))))
        return r, n2.value

    def damage_gradient(self, stream=None, precision="fp64"):
        dev = self.workspace.device
        F = torch.empty(self.n_nodes, dtype=torch.float64, device=dev)
        Phi = torch.empty_like(F)
        act = torch.empty(self.n_nodes, dtype=torch.uint8, device=dev)
        n2 = C.c_double()
        prec = B.PF_MIXED if precision == "mixed" else B.PF_FP64
        B.check(self.lib.pf_op_damage_gradient(self.h, prec, _ptr(F), _ptr(Phi), _ptr(act),
                                               C.byref(n2), C.c_void_p(_stream(stream))))
        return F, Phi, act, n2.value

    def damage_apply(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        prec = B.PF_FP64 if x.dtype == torch.float64 else B.PF_MIXED
        x = x.contiguous()
        y = torch.empty_like(x)
        B.check(self.lib.pf_op_damage_apply(self.h, prec, _ptr(x), _ptr(y),
                                            C.c_void_p(_stream(stream))))
        return y

    def coupling_apply(self, x: torch.Tensor, transpose: bool = False, stream=None) -> torch.Tensor:
        """y = B x (x: n damage values -> 2n displacement values) or B^T x (2n -> n), FP64."""
        x = x.to(torch.float64).contiguous()
        n = self.n_nodes
        y = torch.empty(n if transpose else 2 * n, dtype=torch.float64, device=x.device)
        B.check(self.lib.pf_op_coupling_apply(self.h, 1 if transpose else 0, _ptr(x), _ptr(y),
                                              C.c_void_p(_stream(stream))))
        return y

    def u_solve(self, opts=None, stream=None):
        o = opts or make_opts()
        rep = B.pf_step_report()
        B.check(self.lib.pf_op_u_solve(self.h, C.byref(o), C.c_void_p(_stream(stream)),
                                       C.byref(rep)))
        return rep.as_dict()

    def alpha_solve(self, opts=None, stream=None):
        o = opts or make_opts()
        rep = B.pf_step_report()
        B.check(self.lib.pf_op_alpha_solve(self.h, C.byref(o), C.c_void_p(_stream(stream)),
                                           C.byref(rep)))
        return rep.as_dict()

    def full_residual(self, stream=None):
        v = C.c_double()
        B.check(self.lib.pf_op_full_residual(self.h, C.byref(v), C.c_void_p(_stream(stream))))
        return v.value


def solve_batch(sims, loads, opts=None, stream=None, ctx: Context | None = None):
    lib = B.load()
    n = len(sims)
    ctx = ctx or sims[0].ctx
    hs = (C.c_void_p * n)(*[s.h.value for s in sims])
    ls = (B.pf_load * n)(*[B.pf_load(t, dT) for (t, dT) in loads])
    reps = (B.pf_step_report * n)()
    o = opts or make_opts()
    st = lib.pf_solve_batch(ctx.h, hs, ls, n, C.byref(o), C.c_void_p(_stream(stream)), reps)
    return st, [r.as_dict() for r in reps]


class Server:
    """Serving loop of libpf (pf_server_*): jobs arrive over time, are admitted by HBM footprint
    into one device arena and advance one load step at a time on `workers` host threads, each
    with its own CUDA stream.  Argument marshalling only."""

    def __init__(self, arena_bytes: int, workers: int = 8, ctx: Context | None = None):
        self.lib = B.load()
        self.ctx = ctx or Context(0)
        self.arena = torch.empty(arena_bytes + 256, dtype=torch.uint8,
                                 device=f"cuda:{self.ctx.device}")
        aligned = (self.arena.data_ptr() + 255) & ~255
        h = C.c_void_p()
        B.check(self.lib.pf_server_create(self.ctx.h, C.c_void_p(aligned), arena_bytes, workers,
                                          C.byref(h)))
        self.h = h
        self._jobs = {}

    @staticmethod
    def footprint(w) -> int:
        return B.load().pf_workspace_bytes(C.byref(mesh_desc(w)), B.PF_FP64)

    def now(self) -> float:
        return self.lib.pf_server_now(self.h)

    def submit(self, w, loads=None, opts=None, arrival: float = -1.0, fields: bool = True) -> int:
        """Queue workload w with its load steps (default w.loads); arrival in seconds on the
        server clock (< 0: now).  Returns the job id."""
        loads = list(w.loads if loads is None else loads)
        n = w.n_nodes()
        keep = {
            "loads": (B.pf_load * len(loads))(*[B.pf_load(t, dT) for (t, dT) in loads]),
            "reports": (B.pf_step_report * len(loads))(),
            "latency": (C.c_double * len(loads))(),
            "u": (C.c_double * (2 * n))() if fields else None,
            "alpha": (C.c_double * n)() if fields else None,
            "n": n,
        }
        job = B.pf_job()
        job.mesh = mesh_desc(w)
        job.material = material(w)
        job.loads = C.cast(keep["loads"], C.POINTER(B.pf_load))
        job.n_loads = len(loads)
        job.opts = opts or make_opts(omega=w.omega)
        job.arrival = arrival
        dp = C.POINTER(C.c_double)
        job.u_out = C.cast(keep["u"], dp) if fields else dp()
        job.alpha_out = C.cast(keep["alpha"], dp) if fields else dp()
        job.reports = C.cast(keep["reports"], C.POINTER(B.pf_step_report))
        job.step_latency = C.cast(keep["latency"], dp)
        jid = C.c_int64()
        B.check(self.lib.pf_server_submit(self.h, C.byref(job), C.byref(jid)))
        self._jobs[jid.value] = keep
        return jid.value

    def wait(self, jid: int) -> dict:
        info = B.pf_job_info()
        B.check(self.lib.pf_server_wait(self.h, jid, C.byref(info)))
        k = self._jobs[jid]
        out = {f: getattr(info, f) for f, _ in info._fields_}
        out["reports"] = [r.as_dict() for r in k["reports"]][: info.steps_done]
        out["latency"] = np.array(k["latency"][: info.steps_done])
        if k["u"] is not None:
            out["u"] = np.array(k["u"]).reshape(k["n"], 2)
            out["alpha"] = np.array(k["alpha"])
        return out

    def drain(self):
        B.check(self.lib.pf_server_drain(self.h))

    def stats(self) -> dict:
        s = B.pf_server_stats()
        B.check(self.lib.pf_server_get_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.pf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
