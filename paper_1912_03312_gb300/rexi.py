"""Python front end of the REXI engine: thin wrappers over the C ABI.

PyTorch supplies device memory and streams only; every step of the method runs
in the library's CUDA kernels.  State vectors are ``torch.complex128`` CUDA
tensors shaped like the grid (numpy order: (N_z, N_y, N_x), x fastest).
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _check_state(t, n, name):
    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda:
        raise TypeError("%s must be a complex128 CUDA tensor" % name)
    if t.numel() != n or not t.is_contiguous():
        raise ValueError("%s must be contiguous with %d elements" % (name, n))


def options(precision="mixed", restart=None, max_iters=2000, tol=0.0, inner_tol=1e-5, R1=0.0,
            eps_target=1e-9, allow_substeps=True, stabilize_eps=0.0, want_backward=False, device=-1,
            shared_first_cycle=True, ortho="dcgs2", window=0):
    """Plan options (``rexi_options``).  ``restart`` is the GMRES restart length
    (default 30), or with ``ortho="lanczos"`` the largest Krylov dimension of a
    substep's shared basis (default 256; there are no restarts).  ``precision``:
    "mixed" (c64 Krylov work with FP64 refinement), "fp64", or "df64" (Lanczos
    only: the recurrence in double-float pairs on the FP32 pipe)."""
    if restart is None:
        restart = 256 if ortho == "lanczos" else 30
    o = N.Options()
    N.load().rexi_options_default(C.byref(o))
    if precision not in ("mixed", "fp64", "df64"):
        raise ValueError("precision must be 'mixed', 'fp64' or 'df64'")
    o.precision = {"mixed": N.REXI_MIXED, "fp64": N.REXI_FP64, "df64": N.REXI_DF64}[precision]
    o.restart_m = int(restart)
    o.max_iters = int(max_iters)
    o.tol = float(tol)
    o.inner_tol = float(inner_tol)
    o.R1 = float(R1)
    o.eps_target = float(eps_target)
    o.allow_substeps = 1 if allow_substeps else 0
    o.stabilize_eps = float(stabilize_eps)
    o.want_backward = 1 if want_backward else 0
    o.device = int(device)
    o.shared_first_cycle = 1 if shared_first_cycle else 0
    if ortho not in ("dcgs2", "cgs2", "lanczos"):
        raise ValueError("ortho must be 'dcgs2', 'cgs2' or 'lanczos'")
    o.ortho = {"cgs2": 0, "dcgs2": 1, "lanczos": 2}[ortho]
    o.window = int(window)
    return o


def fcf(K, R1=0.0, eps_target=1e-9):
    """FCF poles/weights of exp on i[-R1, R1] (host, double-double):
    returns (sigma, beta, info) with complex128 numpy arrays."""
    lib = N.load()
    s = (C.c_double * (2 * K))()
    b = (C.c_double * (2 * K))()
    R = C.c_double()
    sk1 = C.c_double()
    mre = C.c_double()
    amp = C.c_double()
    N.check(lib.rexi_fcf(int(K), float(R1), float(eps_target), s, b, C.byref(R), C.byref(sk1),
                         C.byref(mre), C.byref(amp)), "rexi_fcf")
    sa = np.array(s[:]).view(np.complex128)
    ba = np.array(b[:]).view(np.complex128)
    return sa, ba, {"R1": R.value, "sigma_K1": sk1.value, "min_re_sigma": mre.value,
                    "amplification": amp.value}


def stats_dict(st, K):
    return {"status": st.status, "n_sub": st.n_sub, "max_iters_seen": st.max_iters_seen,
            "total_iters": st.total_iters, "total_cycles": st.total_cycles,
            "iters": list(st.iters[:K]), "cycles": list(st.cycles[:K]), "iters_sq": list(st.iters_sq[:K]),
            "resid": list(st.resid[:K]), "bytes": st.bytes, "flops64": st.flops64, "ops32": st.ops32}


class Plan:
    """One problem: grid, potential, step dt and K poles (``rexi_plan_create``)."""

    def __init__(self, n, lo, hi, V, dt, K, hbar=1.0, mass=1.0, **opts):
        lib = N.load()
        n = tuple(int(v) for v in n)
        self.shape = tuple(reversed(n))
        self.n = int(np.prod(n))
        g = N.Grid()
        g.ndim = len(n)
        for d in range(len(n)):
            g.n[d] = n[d]
            g.lo[d] = float(lo[d])
            g.hi[d] = float(hi[d])
        g.hbar = float(hbar)
        g.mass = float(mass)
        Vh = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
        if Vh.size != self.n:
            raise ValueError("V has %d entries, grid has %d" % (Vh.size, self.n))
        self.opts = options(**opts)
        self._h = C.c_void_p()
        self.K = int(K)
        rc = lib.rexi_plan_create(C.byref(self._h), C.byref(g), Vh.ctypes.data_as(C.POINTER(C.c_double)),
                                  float(dt), self.K, C.byref(self.opts))
        N.check(rc, "rexi_plan_create")
        self.create_status = rc
        self.grid = g

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                N.load().rexi_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self):
        return self._h

    def info(self):
        i = N.PlanInfo()
        N.check(N.load().rexi_plan_get_info(self._h, C.byref(i)), "rexi_plan_get_info")
        return {f: getattr(i, f) for f, _ in N.PlanInfo._fields_}

    def poles(self):
        K = self.K
        z = (C.c_double * (2 * K))()
        a = (C.c_double * (2 * K))()
        a0 = (C.c_double * 2)()
        ns = C.c_int()
        N.check(N.load().rexi_plan_poles(self._h, z, a, a0, C.byref(ns)), "rexi_plan_poles")
        return (np.array(z[:]).view(np.complex128), np.array(a[:]).view(np.complex128),
                complex(a0[0], a0[1]), ns.value)

    def fcf(self):
        K = self.K
        s = (C.c_double * (2 * K))()
        b = (C.c_double * (2 * K))()
        N.check(N.load().rexi_plan_fcf(self._h, s, b), "rexi_plan_fcf")
        return np.array(s[:]).view(np.complex128), np.array(b[:]).view(np.complex128)

    def set_potential(self, V, stream=None):
        """Replace V (CUDA float64 tensor or numpy array), keeping poles and substeps."""
        if isinstance(V, torch.Tensor) and V.is_cuda:
            Vt = V.detach().to(torch.float64).contiguous()
            rc = N.load().rexi_plan_set_potential(self._h, _ptr(Vt), 1, _stream_handle(stream))
        else:
            Vh = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
            rc = N.load().rexi_plan_set_potential(self._h, C.c_void_p(Vh.ctypes.data), 0,
                                                  _stream_handle(stream))
        return N.check(rc, "rexi_plan_set_potential")

    def step(self, psi, out=None, stream=None, stats=False):
        """One user step dt on the device.  Returns out (and a stats dict)."""
        _check_state(psi, self.n, "psi")
        if out is None:
            out = torch.empty_like(psi)
        _check_state(out, self.n, "out")
        st = N.Stats() if stats else None
        rc = N.load().rexi_step(self._h, _ptr(psi), _ptr(out), _stream_handle(stream),
                                C.byref(st) if st is not None else None)
        N.check(rc, "rexi_step")
        return (out, stats_dict(st, self.K)) if stats else out

    def step_host(self, psi_host, out_host=None, stream=None):
        """One step through host buffers (complex128 numpy arrays; pinned tensors also work)."""
        if isinstance(psi_host, torch.Tensor):
            src = psi_host
            dst = out_host if out_host is not None else torch.empty_like(psi_host)
            ps, pd = src.data_ptr(), dst.data_ptr()
        else:
            src = np.ascontiguousarray(psi_host, dtype=np.complex128)
            dst = out_host if out_host is not None else np.empty_like(src)
            ps, pd = src.ctypes.data, dst.ctypes.data
        rc = N.load().rexi_step_host(self._h, C.c_void_p(ps), C.c_void_p(pd), _stream_handle(stream), None)
        N.check(rc, "rexi_step_host")
        return dst

    def cheb_step(self, psi, out=None, tol=0.0, stream=None):
        """One step dt by the Chebyshev propagator of Sec. 4 (``rexi_cheb_step``):
        returns (out, degree)."""
        _check_state(psi, self.n, "psi")
        if out is None:
            out = torch.empty_like(psi)
        _check_state(out, self.n, "out")
        deg = C.c_int(0)
        N.check(N.load().rexi_cheb_step(self._h, _ptr(psi), _ptr(out), float(tol), _stream_handle(stream),
                                        C.byref(deg)), "rexi_cheb_step")
        return out, deg.value

    def solve_poles(self, b, stream=None, stats=False):
        """x_k = (tau H - z_k)^{-1} b for every pole: (K, *shape) complex128."""
        _check_state(b, self.n, "b")
        x = torch.empty((self.K,) + self.shape, dtype=torch.complex128, device=b.device)
        st = N.Stats() if stats else None
        rc = N.load().rexi_solve_poles(self._h, _ptr(b), _ptr(x), _stream_handle(stream),
                                       C.byref(st) if st is not None else None)
        N.check(rc, "rexi_solve_poles")
        return (x, stats_dict(st, self.K)) if stats else x

    def apply_poles(self, v, stream=None):
        """w_k = (tau H - z_k) v_k for v of shape (K, *shape)."""
        if v.dtype != torch.complex128 or not v.is_cuda or v.numel() != self.K * self.n or not v.is_contiguous():
            raise ValueError("v must be a contiguous complex128 CUDA tensor of K*n elements")
        w = torch.empty_like(v)
        N.check(N.load().rexi_apply_poles(self._h, _ptr(v), _ptr(w), _stream_handle(stream)), "rexi_apply_poles")
        return w

    def pole_sum(self, psi, x, stream=None):
        """alpha_0 psi + sum_k alpha_k x_k."""
        _check_state(psi, self.n, "psi")
        out = torch.empty_like(psi)
        N.check(N.load().rexi_pole_sum(self._h, _ptr(psi), _ptr(x.contiguous()), _ptr(out),
                                       _stream_handle(stream)), "rexi_pole_sum")
        return out

    def step_backward(self, psi_n, grad_out, dLdV, grad_in=None, stream=None, stats=False):
        """Vector-Jacobian product of one step (see rexi.h); dLdV is accumulated."""
        _check_state(psi_n, self.n, "psi_n")
        _check_state(grad_out, self.n, "grad_out")
        if grad_in is None:
            grad_in = torch.empty_like(grad_out)
        if dLdV.dtype != torch.float64 or not dLdV.is_cuda or dLdV.numel() != self.n:
            raise ValueError("dLdV must be a float64 CUDA tensor with n entries")
        st = N.Stats() if stats else None
        rc = N.load().rexi_step_backward(self._h, _ptr(psi_n), _ptr(grad_out), _ptr(grad_in), _ptr(dLdV),
                                         _stream_handle(stream), C.byref(st) if st is not None else None)
        N.check(rc, "rexi_step_backward")
        return (grad_in, stats_dict(st, self.K)) if stats else grad_in

    def last_status(self):
        return N.load().rexi_plan_last_status(self._h)

    def last_work(self):
        """(bytes, FP64 flops) the last launch counted (``rexi_plan_last_work``)."""
        b, f = C.c_double(0.0), C.c_double(0.0)
        N.check(N.load().rexi_plan_last_work(self._h, C.byref(b), C.byref(f)), "rexi_plan_last_work")
        return b.value, f.value

    def last_launches(self):
        return N.load().rexi_plan_last_launches(self._h)

    PHASES = {0: "substep start", 1: "FP64 residual", 2: "cycle decision", 3: "matvec + dot sweep 1",
              4: "CGS sweep 2", 5: "CGS update", 6: "Givens", 7: "x update", 8: "pole sum",
              9: "DCGS2 matvec + dots", 10: "DCGS2 update + Givens", 11: "Lanczos sweep",
              12: "Lanczos back substitution", 13: "Lanczos pole sum", 99: "launch"}

    def set_timeout(self, seconds=0.0):
        """Limit of every device-side wait (``rexi_plan_set_timeout``; <= 0: the 4 s default)."""
        N.check(N.load().rexi_plan_set_timeout(self._h, float(seconds)), "rexi_plan_set_timeout")

    def set_trace(self, capacity=65536):
        N.check(N.load().rexi_plan_set_trace(self._h, int(capacity)), "rexi_plan_set_trace")

    def read_trace(self):
        """[(phase code, seconds since the launch started)] of the last launch."""
        cap = 1 << 16
        buf = (C.c_longlong * (2 * cap))()
        cnt = N.check(N.load().rexi_plan_read_trace(self._h, buf, cap), "rexi_plan_read_trace")
        cnt = min(cnt, cap)
        rec = [(int(buf[2 * i]), int(buf[2 * i + 1])) for i in range(cnt)]
        if not rec:
            return []
        t0 = rec[0][1]
        return [(c, (t - t0) * 1e-9) for c, t in rec]

    def set_cta_trace(self, phases=4096):
        """Record every CTA's arrival at the first `phases` barriers (0 disables)."""
        N.check(N.load().rexi_plan_set_cta_trace(self._h, int(phases)), "rexi_plan_set_cta_trace")

    def read_cta_trace(self):
        """Arrival times (ns, int64 array [barriers, grid]) of the last launch."""
        lib = N.load()
        g = C.c_int(0)
        cnt = N.check(lib.rexi_plan_read_cta_trace(self._h, None, 0, C.byref(g)), "rexi_plan_read_cta_trace")
        if cnt <= 0 or g.value <= 0:
            return np.zeros((0, max(g.value, 0)), dtype=np.int64)
        buf = np.zeros(cnt * g.value, dtype=np.int64)
        ptr = buf.ctypes.data_as(C.POINTER(C.c_longlong))
        cnt2 = N.check(lib.rexi_plan_read_cta_trace(self._h, ptr, buf.size, C.byref(g)), "rexi_plan_read_cta_trace")
        rows = min(cnt, cnt2, buf.size // g.value)
        return buf[:rows * g.value].reshape(rows, g.value)

    def balance_summary(self):
        """Per phase kind, from the phase and CTA traces of the last launch:
        (count, mean phase seconds, mean seconds until the first CTA arrived,
        mean seconds until the last CTA arrived, mean barrier release latency)."""
        lib = N.load()
        cap = 1 << 16
        buf = (C.c_longlong * (2 * cap))()
        cnt = min(N.check(lib.rexi_plan_read_trace(self._h, buf, cap), "rexi_plan_read_trace"), cap)
        rec = [(int(buf[2 * i]), int(buf[2 * i + 1])) for i in range(cnt)]
        arr = self.read_cta_trace()
        out = {}
        for r in range(1, min(len(rec), arr.shape[0])):
            start, (code, release) = rec[r - 1][1], rec[r]
            a = arr[r]
            name = self.PHASES.get(code, str(code))
            v = out.setdefault(name, [0, 0.0, 0.0, 0.0, 0.0])
            v[0] += 1
            v[1] += (release - start) * 1e-9
            v[2] += (a.min() - start) * 1e-9
            v[3] += (a.max() - start) * 1e-9
            v[4] += (release - a.max()) * 1e-9
        return {k: (v[0], v[1] / v[0], v[2] / v[0], v[3] / v[0], v[4] / v[0]) for k, v in out.items()}

    def trace_summary(self):
        """Total seconds and count per phase of the last launch."""
        rec = self.read_trace()
        out = {}
        for (c0, t0), (c1, t1) in zip(rec, rec[1:]):
            name = self.PHASES.get(c1, str(c1))
            tot, cnt = out.get(name, (0.0, 0))
            out[name] = (tot + (t1 - t0), cnt + 1)
        return out


def step_batched(plans, psis, outs=None, stream=None, stats=False):
    """One step of every problem in one persistent launch (``rexi_step_batched``)."""
    B = len(plans)
    if outs is None:
        outs = [torch.empty_like(p) for p in psis]
    for pl, a, b in zip(plans, psis, outs):
        _check_state(a, pl.n, "psi")
        _check_state(b, pl.n, "out")
    H = (C.c_void_p * B)(*[pl.handle.value for pl in plans])
    I = (C.c_void_p * B)(*[a.data_ptr() for a in psis])
    O = (C.c_void_p * B)(*[b.data_ptr() for b in outs])
    st = (N.Stats * B)() if stats else None
    rc = N.load().rexi_step_batched(H, B, I, O, _stream_handle(stream), st)
    N.check(rc, "rexi_step_batched")
    if stats:
        return outs, [stats_dict(st[b], plans[b].K) for b in range(B)]
    return outs


class RexiEvolve(torch.autograd.Function):
    """psi(T) = S(V)^nsteps psi0 with dL/dV and dL/dpsi0 by adjoint shifted solves.

    Forward keeps the state before every user step (checkpoints); backward runs
    ``rexi_step_backward`` from the last step to the first.  The plan's poles,
    centre and substeps stay fixed while V changes (``set_potential``).
    """

    @staticmethod
    def forward(ctx, V, psi0, plan, nsteps):
        plan.set_potential(V)
        states = [psi0.detach().contiguous()]
        cur = states[0]
        for _ in range(int(nsteps)):
            cur = plan.step(cur)
            states.append(cur)
        ctx.plan = plan
        ctx.states = states[:-1]
        ctx.Vshape = V.shape
        return states[-1]

    @staticmethod
    def backward(ctx, grad_out):
        plan = ctx.plan
        G = grad_out.contiguous().to(torch.complex128)
        dV = torch.zeros(plan.n, dtype=torch.float64, device=G.device)
        for psi_n in reversed(ctx.states):
            G = plan.step_backward(psi_n, G, dV)
        return dV.reshape(ctx.Vshape), G, None, None
