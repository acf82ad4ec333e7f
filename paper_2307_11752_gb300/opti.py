"""Adjoint-driven optimisation of the porosity field (the guide's chapter
"Optimization" and its example domainIdentification3d) and of the force field
(example testFlowOpti3d, adjoint variant: three control components per cell).

A control alpha lives on the cells of a design domain; the porosity there is
gamma = p(alpha) for a projection p onto [0, 1] (section "Optimizer Classes",
"smooth projection map"), and gamma keeps its given values elsewhere.  The
objective J(gamma) and dJ/dgamma come from a differentiable ``evaluate`` -- on
the GPU that is :func:`paper_2307_11752_gb300.olb.velocity_misfit_loss`, whose
backward pass is the discrete adjoint of ``olb_adjoint_run_misfit``.  The descent
is torch's L-BFGS with a strong Wolfe line search, in place of the guide's LBFGS
optimiser with its "StrongWolfe" step condition (sections "Descent Algorithms",
"Step Size Algorithms").
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List

PROJECTIONS = ("sigmoid", "rectifier")


def project(alpha, name: str):
    """gamma = p(alpha).  sigmoid: 1 / (1 + exp(-alpha)), smooth onto (0, 1);
    rectifier: alpha clamped to [0, 1] (gradient 0 outside)."""
    import torch

    if name == "sigmoid":
        return torch.sigmoid(alpha)
    if name == "rectifier":
        return alpha.clamp(0.0, 1.0)
    raise ValueError(f"unknown projection {name!r} (expected one of {PROJECTIONS})")


def unproject(gamma, name: str):
    """alpha with p(alpha) = gamma (gamma clipped into the open interval for sigmoid)."""
    import torch

    if name == "sigmoid":
        g = gamma.clamp(1e-6, 1.0 - 1e-6)
        return torch.log(g / (1.0 - g))
    if name == "rectifier":
        return gamma.clone()
    raise ValueError(f"unknown projection {name!r} (expected one of {PROJECTIONS})")


@dataclass
class Result:
    alpha: object                 # control on the design cells (1-d tensor)
    gamma: object                 # full porosity field [nz, ny, nx]
    # J and |dJ/dalpha| at the start of each L-BFGS iteration, then at the final control
    objective: List[float] = field(default_factory=list)
    gradient_norm: List[float] = field(default_factory=list)
    evaluations: int = 0          # calls of evaluate (line-search trials included)


def identify_porosity(evaluate: Callable, gamma_fixed, design, gamma_start, projection: str = "sigmoid",
                      iterations: int = 20, history_size: int = 10, tolerance: float = 0.0,
                      line_search_evaluations: int = 25) -> Result:
    """Minimise J(gamma) over the porosity of the design cells.

    evaluate     gamma (float64 tensor [nz, ny, nx]) -> 0-d tensor J, differentiable in gamma
    gamma_fixed  porosity outside the design domain (float64 tensor [nz, ny, nx])
    design       bool tensor [nz, ny, nx], the design domain
    gamma_start  initial porosity of the design cells (float or tensor broadcastable to them)
    iterations   L-BFGS iterations (each runs one or more evaluations in its line search)
    tolerance    stop once J falls to or below this value
    line_search_evaluations  evaluations allowed per iteration.  The line search
                 starts from a step of |dJ/dalpha| and may need many trials to grow
                 to the minimiser along the direction; torch's default for one
                 iteration per call (5/4 of it, i.e. 1) would cut it off at the first.
    """
    import torch

    design = design.to(device=gamma_fixed.device, dtype=torch.bool)
    if int(design.sum()) == 0:
        raise ValueError("the design domain holds no cell")
    g0 = torch.as_tensor(gamma_start, dtype=torch.float64, device=gamma_fixed.device)
    g0 = g0.expand_as(gamma_fixed)[design] if g0.dim() else g0.expand(int(design.sum()))
    alpha = unproject(g0.clone(), projection).detach().requires_grad_(True)
    res = Result(alpha=alpha, gamma=None)

    def compose(a):
        g = gamma_fixed.clone()
        g[design] = project(a, projection)
        return g

    opt = torch.optim.LBFGS([alpha], lr=1.0, max_iter=1, max_eval=line_search_evaluations,
                            history_size=history_size, line_search_fn="strong_wolfe", tolerance_grad=0.0,
                            tolerance_change=0.0)

    record = [False]  # the next evaluation is the first of an iteration

    def closure():
        opt.zero_grad()
        J = evaluate(compose(alpha))
        J.backward()
        res.evaluations += 1
        if record[0]:
            res.objective.append(float(J.detach()))
            res.gradient_norm.append(float(alpha.grad.norm()))
            record[0] = False
        return J

    for _ in range(iterations):
        record[0] = True
        opt.step(closure)
        if res.objective[-1] <= tolerance:
            break
    record[0] = True
    closure()  # J at the final control
    with torch.no_grad():
        res.gamma = compose(alpha)
    return res


def identify_force(evaluate: Callable, force_fixed, design, force_start=0.0, iterations: int = 20,
                   history_size: int = 10, tolerance: float = 0.0, line_search_evaluations: int = 25) -> Result:
    """Minimise J(F) over the force density of the design cells: the control is the
    distributed field, a force vector per design cell (testFlowOpti3d with the adjoint
    LBM).  No projection: the force is unconstrained.

    evaluate     F (float64 tensor [3, nz, ny, nx]) -> 0-d tensor J, differentiable in F
                 (on the GPU: :func:`paper_2307_11752_gb300.olb.force_misfit_loss`)
    force_fixed  force density outside the design domain ([3, nz, ny, nx])
    design       bool tensor [nz, ny, nx]
    force_start  initial force of the design cells (float, or tensor broadcastable
                 to [3, n_design])
    Returns a Result whose ``alpha`` is the control [3, n_design] and whose ``gamma``
    field holds the identified force density [3, nz, ny, nx]."""
    import torch

    design = design.to(device=force_fixed.device, dtype=torch.bool)
    nd = int(design.sum())
    if nd == 0:
        raise ValueError("the design domain holds no cell")
    start = torch.as_tensor(force_start, dtype=torch.float64, device=force_fixed.device)
    control = start.expand(3, nd).clone().detach().requires_grad_(True)
    res = Result(alpha=control, gamma=None)

    def compose(c):
        F = force_fixed.clone()
        F[:, design] = c
        return F

    opt = torch.optim.LBFGS([control], lr=1.0, max_iter=1, max_eval=line_search_evaluations,
                            history_size=history_size, line_search_fn="strong_wolfe", tolerance_grad=0.0,
                            tolerance_change=0.0)
    record = [False]

    def closure():
        opt.zero_grad()
        J = evaluate(compose(control))
        J.backward()
        res.evaluations += 1
        if record[0]:
            res.objective.append(float(J.detach()))
            res.gradient_norm.append(float(control.grad.norm()))
            record[0] = False
        return J

    for _ in range(iterations):
        record[0] = True
        opt.step(closure)
        if res.objective[-1] <= tolerance:
            break
    record[0] = True
    closure()
    with torch.no_grad():
        res.gamma = compose(control)
    return res
