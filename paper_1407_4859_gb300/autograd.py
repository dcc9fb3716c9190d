"""Differentiation through layout changes and chains of fp32 sections.

State in a layout is a list of float32 tensors, one (n, k) tensor per group of k fields (all fields
fp32, so a group's struct is k contiguous floats).  Three autograd Functions:

* RemapFn: moves the groups that change from one layout to another with the remap kernel; its
  backward is the inverse remap of the incoming gradients (the same byte permutation, reversed).
  Groups the two layouts share are not inputs or outputs of the Function: the same tensor carries
  the data and its gradient straight through.
* SegmentFn: runs a run of axpb / mul / tanh sections in place in one layout, saving each value a
  section overwrites; its backward walks the sections in reverse with the adjoint kernel
  (adha_section_backward), which restores the overwritten field and propagates the adjoints.
* CopyFn: a copy of the state by the remap kernel, where the first section keeps the input layout.

DifferentiableProgram strings them together for a whole program under a layout plan.  Every
forward and backward step runs in the library's kernels; PyTorch only allocates and orders them.
Memory: the forward keeps one saved field (n floats) per section and every layout's moved groups;
the backward hands the program's state back to what it was before each segment, in place, so the
forward outputs hold the input-side values once backward() has run (copy them first if needed).
"""
import torch

from .api import c_section, adha_remap, adha_run_section, adha_section_backward


def _copy(schema, n, layout, groups):
    """Fresh copies of a layout's group tensors, moved by the library's remap kernel (identical
    groups at different addresses are copied, not aliased)."""
    out = [torch.empty_like(g) for g in groups]
    adha_remap(schema, n, layout, list(groups), layout, out)
    return out


class CopyFn(torch.autograd.Function):
    """A copy of the state (sections then update the copy in place and leave the inputs intact);
    its backward passes the gradients through."""

    @staticmethod
    def forward(ctx, meta, *groups):
        schema, n, layout = meta
        return tuple(_copy(schema, n, layout, groups))

    @staticmethod
    def backward(ctx, *grads):
        return (None,) + grads


def _alias_map(src, dst):
    """dst group index -> src group index for groups identical in both layouts."""
    out = {}
    for d, g in enumerate(dst.groups):
        for s, h in enumerate(src.groups):
            if g == h:
                out[d] = s
    return out


class RemapFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, meta, *moved_src):
        schema, n, src, dst, src_all = meta
        alias = _alias_map(src, dst)
        moved_s = [s for s in range(len(src.groups)) if s not in alias.values()]
        src_ptrs = list(src_all)
        for k, s in enumerate(moved_s):
            src_ptrs[s] = moved_src[k]
        out = {}
        dst_ptrs = []
        for d, g in enumerate(dst.groups):
            if d in alias:
                dst_ptrs.append(src_ptrs[alias[d]])
            else:
                out[d] = torch.empty((n, len(g)), dtype=torch.float32, device="cuda")
                dst_ptrs.append(out[d])
        adha_remap(schema, n, src, src_ptrs, dst, dst_ptrs)
        ctx.meta = (schema, n, src, dst, alias, moved_s)
        return tuple(out[d] for d in sorted(out))

    @staticmethod
    def backward(ctx, *grads):
        schema, n, src, dst, alias, moved_s = ctx.meta
        moved_d = [d for d in range(len(dst.groups)) if d not in alias]
        gd = {}
        for k, d in enumerate(moved_d):
            g = grads[k]
            gd[d] = g.contiguous() if g is not None else torch.zeros((n, len(dst.groups[d])), dtype=torch.float32,
                                                                       device="cuda")
        gs = {s: torch.empty((n, len(src.groups[s])), dtype=torch.float32, device="cuda") for s in moved_s}
        # shared groups: one placeholder buffer on both sides, so the kernel leaves them alone
        placeholder = torch.empty(16, dtype=torch.uint8, device="cuda")
        d_ptrs = [gd[d] if d in gd else placeholder for d in range(len(dst.groups))]
        s_ptrs = []
        for s in range(len(src.groups)):
            if s in gs:
                s_ptrs.append(gs[s])
            else:
                d = [dd for dd, ss in alias.items() if ss == s][0]
                s_ptrs.append(d_ptrs[d])
        adha_remap(schema, n, dst, d_ptrs, src, s_ptrs)      # inverse remap of the gradients
        return (None,) + tuple(gs[s] for s in moved_s)


class SegmentFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, meta, *groups):
        schema, n, layout, sections = meta
        saves = []
        for s in sections:
            cs = c_section(s)
            save = torch.empty(n, dtype=torch.float32, device="cuda")
            adha_run_section(schema, n, layout, list(groups), cs, save=save)
            saves.append((cs, save))
        ctx.meta = (schema, n, layout)
        ctx.state = groups          # updated in place; the backward restores it section by section
        ctx.saves = saves
        ctx.mark_dirty(*groups)
        return groups

    @staticmethod
    def backward(ctx, *grads):
        schema, n, layout = ctx.meta
        # the adjoint kernels update the gradients in place: work on copies of the incoming ones
        g = [x.contiguous() if x is not None else torch.zeros((n, len(layout.groups[k])), dtype=torch.float32,
                                                              device="cuda")
             for k, x in enumerate(grads)]
        g = _copy(schema, n, layout, g)
        for cs, save in reversed(ctx.saves):
            adha_section_backward(schema, n, layout, list(ctx.state), g, cs, save)
        # the state tensors' grad_fn refers to ctx: drop them here, or the step's memory waits for
        # Python's cycle collector
        ctx.saves = None
        ctx.state = None
        return (None,) + tuple(g)


class DifferentiableProgram:
    """A chain of axpb / mul / tanh sections under a layout plan (one Layout per section)."""

    def __init__(self, schema, n, in_layout, sections, plan_layouts):
        for s in sections:
            if s.op not in ("axpb", "mul", "tanh"):
                raise ValueError("differentiable programs take axpb, mul and tanh sections (got %s)" % s.op)
        self.schema, self.n, self.in_layout = schema, n, in_layout
        self.sections = list(sections)
        self.plan = list(plan_layouts)

    def _remap(self, state, src, dst):
        alias = _alias_map(src, dst)
        moved_s = [s for s in range(len(src.groups)) if s not in alias.values()]
        outs = RemapFn.apply((self.schema, self.n, src, dst, list(state)), *[state[s] for s in moved_s])
        it = iter(outs)
        return [state[alias[d]] if d in alias else next(it) for d in range(len(dst.groups))]

    def forward(self, in_groups):
        """in_groups: (n, k) float32 tensors of the input layout.  Returns (final layout, groups)."""
        cur = self.in_layout
        state = list(in_groups)
        first = True
        k = 0
        while k < len(self.sections):
            lay = self.plan[k]
            j = k
            while j < len(self.sections) and self.plan[j] == lay:
                j += 1
            if lay != cur:
                state = self._remap(state, cur, lay)
                cur = lay
            elif first:
                state = list(CopyFn.apply((self.schema, self.n, cur), *state))   # leave the inputs intact
            first = False
            state = list(SegmentFn.apply((self.schema, self.n, cur, self.sections[k:j]), *state))
            k = j
        return cur, state
