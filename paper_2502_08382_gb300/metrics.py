"""Host-side metric helpers (no GPU work).

break_even: the amortisation point of the explicit dual operator (Sec. III):
the number of solver iterations after which assembling F_i explicitly and
applying it beats applying it implicitly,
    n* = ceil((T_prep_explicit - T_prep_implicit) / (T_apply_implicit - T_apply_explicit)).
"""
import math


def break_even(prep_expl, apply_expl, prep_impl, apply_impl):
    """Smallest iteration count at which the explicit approach has paid off.
    Returns None when the explicit apply is not faster than the implicit one."""
    gain = apply_impl - apply_expl
    if gain <= 0:
        return None
    extra = prep_expl - prep_impl
    if extra <= 0:
        return 1
    return int(math.ceil(extra / gain))
