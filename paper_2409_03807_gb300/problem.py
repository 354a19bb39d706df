"""Set up a liblsn context from a synthetic workload (argument marshalling)."""
from ._native import Context


def context_from_problem(p, precision="fp32", device=0, stream=None, tol=None,
                         optimizer="newton", history=10):
    """p is a ``workloads.Problem``; returns a ready ``Context``."""
    c = p.config
    ctx = Context(device, stream)
    ctx.set_mesh(p.X0, p.tets)
    ctx.set_material(c.youngs, c.poisson, c.density, c.gravity)
    if c.cubature > 0:
        ctx.set_cubature(p.cub_idx, p.cub_w)
    ctx.set_constraints(p.cnodes, p.targets(0))
    ctx.set_decoder(p.Ws, p.bs, c.out_scale, precision)
    if getattr(p, "affine_center", None) is not None:
        ctx.set_affine_modes(p.affine_center)
    if getattr(c, "ground_k", 0.0) > 0.0:
        ctx.set_ground(c.ground_h, c.ground_k)
    ctx.set_solver(c.eps if tol is None else tol, c.max_newton, c.max_ls, c.armijo_c)
    if optimizer != "newton":
        ctx.set_optimizer(optimizer, history)
    ctx.set_state(v=getattr(p, "v0", None))
    return ctx
