"""GB300-native FLAPW Hamiltonian / overlap assembly (``libhs``).

For one k-point the library assembles

    H = sum_a A_a^H T^AA_a A_a + A_a^H T^AB_a B_a + B_a^H T^BA_a A_a + B_a^H T^BB_a B_a
    S = sum_a A_a^H A_a + B_a^H U_a^H U_a B_a

(Eqs. (h) and (s)) on an sm_103a GPU, computes the matching coefficients A, B that
enter them (Sec. 1.1), and reduces the generalized eigenproblem H c = lambda S c to
standard form.  The compute path is the C-ABI shared library ``libhs.so`` built
from ``csrc/``; ``paper_1611_00606_gb300.hs`` is its thin ctypes binding.
``synth`` draws seeded synthetic inputs, ``flops`` counts Algorithm 1's work and
``ksplit`` splits one k-point's atoms over the ranks of a process group.
"""
__all__ = ["hs", "synth", "flops", "ksplit"]
