"""Differentiable rollout of the radiation step with checkpointing.

Section 5.2 of the paper points at differentiable solvers; here the gradient
of a loss of the final state (I_N, u_g,N) with respect to the initial
intensity I_0, the initial gas energy u_g,0, the absorption prefactor kappa
and the emission multiplier eta comes from the library's hand-written reverse
pass.  The forward runs nsteps steps through rt_step and keeps (I, u_g) at the
start of every segment of ckpt_every steps; the backward walks the segments in
reverse, and rt_step_adjoint recomputes each segment from its checkpoint
before reversing it.  The last segment runs through rt_step_record, which
keeps its stage states, so the backward reverses it without a recompute
(rt_step_adjoint_recorded) unless the context has served another rollout or
fluid since.  Every step of both passes runs in the CUDA library; this module
only moves tensors.
"""
import torch

from . import RadiationStep


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, I0, ug0, kappa, eta, st, fluid, dt, nsteps, ckpt_every):
        dev = I0.device
        nc = ug0.shape[0]
        kappa = kappa.detach().contiguous()
        eta = eta.detach().contiguous()
        st.set_fluid(fluid["rho"], ug0.detach().contiguous(), fluid["ucon"], kappa, fluid["alpha_s"], eta)
        st.set_intensity(I0.detach().contiguous())
        ck_I, ck_u, segs = [], [], []
        n = 0
        while n < nsteps:
            k = min(ckpt_every, nsteps - n)
            I = torch.empty_like(I0)
            u = torch.empty(nc, dtype=torch.float64, device=dev)
            st.get_intensity(I)
            st.get_ugas(u)
            ck_I.append(I)
            ck_u.append(u)
            if n + k < nsteps:
                st.step(dt, k)
            else:
                ctx.rec_id = st.step_record(dt, k)
            segs.append(k)
            n += k
        IN = torch.empty_like(I0)
        uN = torch.empty(nc, dtype=torch.float64, device=dev)
        st.get_intensity(IN)
        st.get_ugas(uN)
        ctx.fluid_token = st.fluid_token
        ctx.st, ctx.fluid, ctx.dt, ctx.segs, ctx.I_dtype = st, fluid, dt, segs, I0.dtype
        ctx.ck_I, ctx.ck_u, ctx.kappa, ctx.eta, ctx.ug0 = ck_I, ck_u, kappa, eta, ug0.detach()
        return IN, uN

    @staticmethod
    def backward(ctx, gI, gu):
        st, f = ctx.st, ctx.fluid
        # the context may have served another rollout since: restore this one's
        # fluid (which drops the library's recording of the last segment)
        if st.fluid_token is not ctx.fluid_token:
            st.set_fluid(f["rho"], ctx.ug0.contiguous(), f["ucon"], ctx.kappa, f["alpha_s"], ctx.eta)
        recorded = st.rec_id != 0 and st.rec_id == ctx.rec_id
        I_like, u_like = ctx.ck_I[0], ctx.ck_u[0]
        Ib = torch.zeros_like(I_like) if gI is None else gI.to(torch.float64).contiguous().clone()
        ub = torch.zeros_like(u_like) if gu is None else gu.to(torch.float64).contiguous().clone()
        Ib_in = torch.empty_like(Ib)
        ub_in = torch.empty_like(ub)
        kb = torch.zeros_like(u_like)
        eb = torch.zeros_like(u_like)
        for idx in reversed(range(len(ctx.segs))):
            if recorded and idx == len(ctx.segs) - 1:
                st.step_adjoint_recorded(ctx.rec_id, Ib, ub, Ib_in, ub_in, kb, eb)
            else:
                st.step_adjoint(ctx.ck_I[idx], ctx.ck_u[idx], ctx.dt, ctx.segs[idx], Ib, ub, Ib_in, ub_in, kb, eb)
            Ib, Ib_in = Ib_in, Ib
            ub, ub_in = ub_in, ub
        return Ib.to(ctx.I_dtype), ub, kb, eb, None, None, None, None, None


def rollout(st: RadiationStep, fluid: dict, I0, ug0, kappa, eta, nsteps: int, dt: float = None,
            ckpt_every: int = 8):
    """(I_N, u_g,N) after nsteps steps of size dt (None: the cfl bound with
    cfl 0.4) from (I0, ug0), differentiable in I0, ug0, kappa and eta.

    ``st`` is a RadiationStep on flat geometry with FP64 intensities (an FP64
    reverse pass) or FP32 intensities (FP32 per-element arithmetic with FP64
    per-cell sums and FP64 cotangents);
    ``fluid`` holds the device tensors rho, ucon and alpha_s (float64).  The
    library works on the step's stream, so that stream must be the current
    one (the backward runs on the forward's stream).
    """
    import torch
    if torch.cuda.current_stream().cuda_stream != st.stream:
        raise RuntimeError("rollout: the RadiationStep's stream must be the current CUDA stream")
    if dt is None:
        dt = st.cfl_dt(0.4)
    return _Rollout.apply(I0, ug0, kappa, eta, st, fluid, float(dt), int(nsteps), int(ckpt_every))
