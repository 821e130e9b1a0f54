"""CPU oracle for the reciprocal part of Kroneckerised Particle Mesh Ewald.

TEST INFRASTRUCTURE ONLY.  Plain, slow, float64 numpy code written from the
paper's definitions so that the CUDA path can be checked against it.  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it; the library itself never does, and the two share no code.

Modules
-------
bspline  cardinal B-splines M_n, derivatives and the SPME moduli |b(m)|^2.
spme     charge spreading, the reciprocal influence function, FFT convolution
         (classical PME), gathering of potentials / forces, energy and virial.
skp      the paper's Sum-of-Kronecker-Products mesh operator: the two-level SVD
         compression (§2.1.1), circulant synthesis of the real factors (§2.3,
         Eq. VtV) and the reshaped Kronecker mat-vec (Algorithm 2); the
         sinc-quadrature variant (§2.1.2).
ewald    exact reciprocal Ewald sum, real-space sum and self term, used only to
         pin the others.

Conventions used throughout (one cubic box of side L = 2 r_B, centre c_B):
  fractional coordinate  s = (x - c_B)/L + 1/2 in [0, 1)   (reading of §1.2: the
                         period of the lattice sum is 2 r_B, so the paper's
                         x~ = (x - c_B)/r_B is taken over the period 2 r_B)
  mesh coordinate        u = K s in [0, K)
  reciprocal vector      k = m / L,  m in Z^3
  Coulomb constant       1 (energies in e^2/A)
"""
