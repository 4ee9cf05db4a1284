"""Element-wise agreement criteria for the learned initialiser's gradients.

Per parameter tensor T with reference g_ref (max |g_ref| over T = s_T), every
entry must satisfy |g - g_ref| <= atol * s_T + rtol * |g_ref|, and at least
`bulk` of the entries the tighter |g - g_ref| <= bulk_atol * s_T + rtol * |g_ref|.

Against the FP64 reference that rounds every dense-layer operand to bfloat16
(the operand precision the network is specified with), the remaining
differences are FP32 against FP64 accumulation and the activations whose
FP32 and FP64 values straddle a bfloat16 rounding boundary or a ReLU kink;
they grow toward the first layers (measured on five parameter draws: the 95th
percentile of |g - g_ref| / scale at most 1.4e-2, the maximum 2.9e-2, on the
first layers' biases). Against the plain FP64 reference the operand rounding
itself adds up (unit roundoff 2^-9 per operand, about a dozen dense products
between the output and the first layer's gradient): measured 95th percentile
up to 7.6e-2 and maximum 1.1e-1 of a tensor's scale.
"""
import numpy as np

BF16_REF = dict(atol=5e-2, rtol=2e-2, bulk=0.95, bulk_atol=2.5e-2)
FP64_REF = dict(atol=2e-1, rtol=5e-2, bulk=0.95, bulk_atol=1e-1)


def grad_mismatches(g, ref, shapes, atol, rtol, bulk, bulk_atol):
    """Names of the tensors that fail the criterion (empty list = agreement)."""
    bad = []
    at = 0
    for name, shp in shapes:
        size = int(np.prod(shp))
        a, b = g[at:at + size], ref[at:at + size]
        at += size
        s = float(np.abs(b).max())
        if s == 0.0:
            if np.abs(a).max() > 0.0:
                bad.append(name)
            continue
        err = np.abs(a - b)
        if np.any(err > atol * s + rtol * np.abs(b)):
            bad.append(name)
        elif np.mean(err <= bulk_atol * s + rtol * np.abs(b)) < bulk:
            bad.append(name)
    return bad
