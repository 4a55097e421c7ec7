"""FP64 CPU oracle for the Stolt-based ASHRT/AASHRT deblending path.

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct numpy code written
from the thesis (Ibrahim 2015, "Separating simultaneous seismic sources using
robust inversion of Radon and migration operators").  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import it.  The CUDA library never imports, links or calls anything here,
and nothing here imports the CUDA library: the two share no code.

Modules
-------
dft         naive (matrix) discrete Fourier transforms, the F operators.
stolt       Stolt-based ASHRT / AASHRT forward and its exact transpose
            (ch. 5 Eqs ch5_adj_operator / ch5_forward_operator, ch. 6 Eqs
            ch6_adj_operator / ch6_forward_operator), also for traces at
            irregular positions (the x transform as a DFT at the traces).
timedomain  time-domain ASHRT / AASHRT hyperbolic summation (ch. 3 Table
            ch3_table_Radon_operators, ch. 6 Eqs ch6_AASHRT_forward /
            ch6_AASHRT_adjoint); an independent kinematic check and the
            reference of the GPU time-domain pair.
irls        robust l_p-l_q inversion by IRLS with inner CGLS (ch. 4 Eqs
            ch4_cost_fn, equ:10, equ:11, ch4_epcilon_r) and the quality
            measures Q_PD, Q_R (Eqs ch4_Qpd, ch4_Qr).
fista       l2-l1 inversion by FISTA with a power-method step (ch. 6,
            "Sparse inversion", Eq. cost_fn with p = 2, q = 1).
blending    blending, pseudo-deblending (ch. 2 Eqs ch2_blending,
            pseudodeblending_equ) and shot <-> receiver gather sorting.
unet        the warm-start network (no counterpart in the thesis): forward,
            hand-derived backward, MSE, Adam, bfloat16 storage rounding.
"""
