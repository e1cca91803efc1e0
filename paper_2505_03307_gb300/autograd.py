"""PyTorch autograd bridge for gradients of output weights (qx_tape_*).

``RotationCircuit(n, instrs).coeffs(theta, gens, paulis)`` returns the output
weights c_{gens[k]}(paulis[k]) of the circuit whose RX / RY / RZ angles are the
entries of ``theta`` (in instruction order), as a float64 tensor that carries
a gradient.  The forward pass runs libqx's propagation with per-operator
checkpoints; the backward pass hands the incoming gradient (the cotangent a)
to libqx's reverse pass, which returns dL/dtheta for L = sum_k a_k c_k.  Both
passes run entirely in the library's CUDA kernels; this module only moves
arrays.
"""
from __future__ import annotations

import numpy as np
import torch

from . import qx

ROTATIONS = ("RX", "RY", "RZ", "RXX", "RYY", "RZZ", "CRX", "CRY", "CRZ", "CP")


class _Coeffs(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, circ, gens, paulis, ckpt_stride, opts):
        instrs = circ.with_angles(theta.detach().cpu().numpy())
        lo, hi = min(gens), max(gens) + 1
        plan = qx.group_ops(qx.load_circuit(circ.n, instrs))
        tape = qx.Tape(plan, [g - lo for g in gens], paulis, ckpt_stride=ckpt_stride,
                       gens=(lo, hi), **opts)
        ctx.tape = tape
        ctx.positions = circ.positions
        ctx.theta_meta = (theta.dtype, theta.device)
        return torch.from_numpy(tape.values.copy()).to(theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        a = grad_out.detach().to("cpu", torch.float64).numpy()
        g = ctx.tape.backward(a)[ctx.positions]
        dtype, device = ctx.theta_meta
        return torch.from_numpy(g).to(device=device, dtype=dtype), None, None, None, None, None


class RotationCircuit:
    """A circuit whose rotation angles are free parameters.

    instrs: (gate, q0, q1, theta) tuples as in ``qx.load_circuit``; the angles
    of the rotation instructions (RX / RY / RZ and the two-qubit RXX ... CP)
    are taken from ``theta`` in order (``positions`` lists their instruction
    indices)."""

    def __init__(self, n, instrs):
        self.n = int(n)
        self.instrs = list(instrs)
        self.positions = [i for i, ins in enumerate(self.instrs) if ins[0] in ROTATIONS]

    def angles(self, dtype=torch.float64):
        """The angles written in the instruction list, as a tensor."""
        return torch.tensor([self.instrs[i][3] for i in self.positions], dtype=dtype)

    def with_angles(self, theta):
        theta = np.asarray(theta, np.float64).reshape(-1)
        if theta.size != len(self.positions):
            raise ValueError(f"need {len(self.positions)} angles, got {theta.size}")
        out = list(self.instrs)
        for k, i in enumerate(self.positions):
            g, q0, q1, _ = out[i]
            out[i] = (g, q0, q1, float(theta[k]))
        return out

    def coeffs(self, theta, gens, paulis, ckpt_stride=1, **opts):
        """c_{gens[k]}(paulis[k]) after the circuit (gens are absolute
        generator indices j of Z_j); differentiable in theta.  opts go to
        ``qx.make_opts`` (eps, hbm_budget, precision, ...)."""
        gens = [int(g) for g in gens]
        if len(gens) != len(paulis) or not gens:
            raise ValueError("need one generator per query and at least one query")
        return _Coeffs.apply(theta, self, gens, list(paulis), int(ckpt_stride), dict(opts))


def coeffs(theta, n, instrs, gens, paulis, **kw):
    """Functional form of ``RotationCircuit(n, instrs).coeffs(theta, gens, paulis)``."""
    return RotationCircuit(n, instrs).coeffs(theta, gens, paulis, **kw)
