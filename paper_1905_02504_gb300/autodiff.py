"""torch.autograd wrappers of the step and of the outer-shell objective.

StepWindow runs K steps of fixed dt through the C ABI, keeping one checkpoint
(U, phi) per step on the device; its backward walks the steps in reverse and
calls geo_step_adjoint on each checkpoint (the step is recomputed inside the
adjoint call).  For an FP32-bulk mesh the forward steps run in the FP32-bulk
form and the reverse sweep on an FP64 mesh of the same geometry, i.e. the FP64
linearisation of the step about the FP32-bulk trajectory.  OuterBr2 is J = sum over the outer radial faces of phi^2 / A.
Both compute only in the CUDA library; torch provides the tensors.

Stream order: the library enqueues its work on the mesh's stream, torch on its
current stream.  Each call below makes the mesh stream wait for what torch has
queued before handing it tensors, and makes torch's current stream wait for the
mesh stream before torch reads (or reuses the memory of) what the library wrote.
"""
import torch

from . import geomhd


def _mesh_stream(mesh):
    """The torch view of the stream the mesh enqueues on (0: the legacy default)."""
    return torch.cuda.ExternalStream(mesh.stream) if mesh.stream else torch.cuda.default_stream()


def _wait(waiter, producer):
    """Make stream `waiter` wait for the work queued so far on stream `producer`."""
    if waiter.cuda_stream != producer.cuda_stream:
        ev = torch.cuda.Event()
        ev.record(producer)
        waiter.wait_event(ev)


class StepWindow(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, phi, mesh, dt, K):
        U = U.detach().contiguous()
        phi = phi.detach().contiguous()
        ms, cs = _mesh_stream(mesh), torch.cuda.current_stream()
        _wait(ms, cs)
        checkpoints = []
        geomhd.geo_state_upload(mesh.h, U, phi)
        cur_U, cur_phi = U, phi
        for _ in range(K):
            checkpoints.append((cur_U, cur_phi))
            geomhd.geo_step(mesh.h, dt)
            cur_U = torch.empty_like(U)
            cur_phi = torch.empty_like(phi)
            geomhd.geo_state_download(mesh.h, cur_U, cur_phi)
        _wait(cs, ms)
        ctx.mesh, ctx.dt, ctx.checkpoints = mesh, dt, checkpoints
        return cur_U, cur_phi

    @staticmethod
    def backward(ctx, gU, gphi):
        gU = (torch.zeros_like(ctx.checkpoints[0][0]) if gU is None else gU).contiguous()
        gphi = (torch.zeros_like(ctx.checkpoints[0][1]) if gphi is None else gphi).contiguous()
        adj = ctx.mesh.adjoint_mesh()
        ms, cs = _mesh_stream(adj), torch.cuda.current_stream()
        _wait(ms, cs)
        keep = []   # cotangents read by queued adjoint calls stay allocated until cs waits
        for U_s, phi_s in reversed(ctx.checkpoints):
            gU_in = torch.empty_like(gU)
            gphi_in = torch.empty_like(gphi)
            geomhd.geo_step_adjoint(adj.h, ctx.dt, U_s, phi_s, gU, gphi, gU_in, gphi_in)
            keep.append((gU, gphi))
            gU, gphi = gU_in, gphi_in
        _wait(cs, ms)
        del keep
        return gU, gphi, None, None, None


class OuterBr2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, mesh):
        phi = phi.detach().contiguous()
        _wait(_mesh_stream(mesh), torch.cuda.current_stream())
        g = torch.empty_like(phi)   # written on the mesh stream, which the call synchronises
        J = geomhd.geo_outer_Br2(mesh.h, phi, g)
        ctx.save_for_backward(g)
        return torch.tensor(J, dtype=phi.dtype, device=phi.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return g * gJ, None


def step_window(mesh, U, phi, dt, K):
    return StepWindow.apply(U, phi, mesh, dt, K)


def outer_br2(mesh, phi):
    return OuterBr2.apply(phi, mesh)
