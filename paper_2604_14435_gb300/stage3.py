"""One instance split across ranks: the exchange step of Stage III (Sec. 2.3;
Algorithm 1, Step 4c).

Each rank evaluates a contiguous block of the instance's 2P + 1 parameter-
shift evaluations (dvqls_cost_grad_partials), the per-shift sums (T_g, D_g)
of all ranks are added by one SUM allreduce of (2P + 1) x 4 doubles -- the
paper's allreduce of two scalars per evaluated cost -- and every rank then
forms N_g = |T_g|^2, the cost and the gradient on its GPU
(dvqls_combine_partials).  With NCCL between GPUs, or gloo on CPU; no
arithmetic of the method happens here.
"""


def shift_ranges(S, world_size):
    """Contiguous, disjoint ranges [s0, s1) covering 0 .. S-1, one per rank,
    sizes differing by at most one (ranks beyond S get empty ranges)."""
    if S < 1 or world_size < 1:
        raise ValueError("S and world_size must be >= 1")
    base, extra = divmod(S, world_size)
    out, s0 = [], 0
    for r in range(world_size):
        s1 = s0 + base + (1 if r < extra else 0)
        out.append((s0, s1))
        s0 = s1
    return out


def cost_grad_split(lib, ctx, ansatz, alpha, lcu, b, precision, dist, torch, device, group=None):
    """Cost and gradient of one instance whose shifts are shared among the
    ranks of `dist` (an initialised torch.distributed; None: one rank takes
    every shift).  Returns (cost, grad) as tensors on `device`, identical on
    every rank."""
    n, depth = ansatz.n, ansatz.depth
    P = n * (depth + 1)
    S = 2 * P + 1
    rank, ws = (dist.get_rank(group), dist.get_world_size(group)) if dist is not None else (0, 1)
    s0, s1 = shift_ranges(S, ws)[rank]
    part = torch.zeros(S * 4, dtype=torch.float64, device=device)
    if s1 > s0:
        lib.dvqls_cost_grad_partials(ctx, ansatz, alpha, lcu, b, precision, s0, s1, part)
    if dist is not None:
        dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    cost = torch.zeros(1, dtype=torch.float64, device=device)
    grad = torch.zeros(P, dtype=torch.float64, device=device)
    lib.dvqls_combine_partials(ctx, n, depth, part, cost, grad)
    return cost, grad
