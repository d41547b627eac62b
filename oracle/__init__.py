"""Plain, slow, FP64 CPU oracle for the Lanczos/Sternheimer dielectric path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
runs this code.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

The oracle follows the paper's definitions with no blocking, fusion or
reordering beyond what the definitions state, so that each step can be read
against the paper:

* ``pw``        plane-wave sphere, real-space grid, dense Hamiltonian and exact
                diagonalisation (the DFT ground state is an *input* of the
                method; exact diagonalisation stands in for it).
* ``coulomb``   square root of the (spherically truncated) Coulomb kernel.
* ``response``  chi0 by the Adler-Wiser sum over states (Eq. P), its
                Sternheimer form (Eqs. P1, fvpm, P2a, P2), the squared Hermitian
                form at imaginary frequency (Eq. P2+), the model
                polarizability with H -> T (Sec. Dielectric model, Eq.
                model_eq), and the symmetrised dielectric operator (Eq.
                epsilon).
* ``lanczos``   Lanczos recursion with full Gram-Schmidt re-orthogonalisation
                (Sec. Lanczos, Eq. krylov), the inverse in the Lanczos basis,
                and the split over an exact and a model basis (Eq.
                subs_epsilon).
* ``sigma_p``   residue term Sigma^P_e(delta) of Eq. pe: one short Lanczos per
                pole at its real frequency, seeded with v^1/2 |p* e>.
* ``recycle``   the dielectric matrix at imaginary frequencies from one small
                basis per occupied state built from the static solutions
                (Eq. recy_eq).
* ``sigma_c``   the correlation self-energy Sigma^c_e(delta) (Eq. e_c): the
                frequency integral, the Lorentzian analytic term and the
                residue term, by the sum over states and in a basis of fields.
* ``gradient``  derivative of <phi|eps^-1(0)|phi> with respect to V_loc (not in
                the paper; derived by third-order perturbation theory and pinned
                by central finite differences).

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
