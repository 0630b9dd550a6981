"""CPU oracle for the spin-adapted DMRG / CAS-SCF hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2503_20700_gb300``) never imports it and
shares no code with it.

The oracle is plain, slow, float64 numpy/scipy code written from the paper:

* ``fock``   -- Fock space of n spatial orbitals in site-interleaved
  Jordan-Wigner order, with index maps for E_pq = sum_s a+_ps a_qs and the
  total-spin raising operator S+.
* ``fci``    -- the Hamiltonian of Sec. II.A (one- and two-electron integrals)
  applied to full-space vectors; exact diagonalisation (FCI) with spin
  projection.  This is the exact answer DMRG reaches at untruncated D.
* ``su2``    -- Clebsch-Gordan coefficients from the Racah closed form.
* ``dmrg``   -- two-site DMRG as a variational subspace method (Sec. II.B):
  every block basis is kept as explicit full-space vectors, the effective
  Hamiltonian is the projection of H onto the two-site subspace, and the
  truncation keeps D SU(2) multiplets (Sec. II.C) found from the spin
  operators of the block.  No recoupling coefficients are used.
* ``rdm``    -- spin-free one- and two-particle RDMs (Eqs. onerdm/twordm) and
  their spin-coupled forms (Eq. rdm1_su2 and the two-channel 2-RDM).
* ``casscf`` -- orbital rotation U = exp(-kappa), integral transformation,
  the CAS-SCF energy functional and its orbital gradient (Sec. II.A).
* ``orbital`` -- one- and two-orbital reduced density matrices, orbital
  entropies, mutual information and the Fiedler ordering of the orbitals
  (Sec. II "Numerical procedure", the ordering step).

The kernel-level tests (grouped GEMM, fused sector contraction, eigensolver)
compare against the plain definition written inline in the test (a numpy
matrix product or ``numpy.linalg.eigh``).
"""
