"""Plain FP64 CPU oracle of the Calderón-preconditioned PMCHWT hot path.

TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import, call, link or run anything in this package. The
CUDA library never calls into it, and this package shares no code, header,
table or helper with the CUDA library: the only common input is the seeded
mesh generator ``paper_2008_04772_gb300.meshgen`` (geometry, no method
arithmetic).

It follows Kleanthous, Betcke, Hewett, Escapil-Inchauspé, Jerez-Hanckes and
Baran, "Accelerated Calderón preconditioning for Maxwell transmission
problems" (arXiv 2008.04772), step by step, in the paper's notation:

* ``quadrature``  Gauss–Legendre (Golub–Welsch) and symmetric triangle rules
  (Section 3.3: (q_near, q_medium, q_far) = (4,3,2) gives 36 evaluations per
  regular pair with the 6-point rule; q = 1 gives 1).
* ``spaces``      primal edges, RWG functions (Section 3.2), barycentric
  refinement and Buffa–Christiansen functions (Section 3.2), support boxes.
* ``orc_bem.c``   Galerkin integrals of the electric (S) and magnetic (C)
  boundary operators on a triangle pair (Section 2, eqs. BIOrelns and the
  potentials), regular tensor Gauss rule and Sauter–Schwab singular rules
  (Section 3.3), written straight from the integrand, no moment algebra.
* ``bem``         dense assembly of S, C on RWG or BC spaces; near-field
  cutoff (eq. nf_condition read at entry level); Gram matrices (eqs. MassA,
  MassP).
* ``pmchwt``      the block system (eqs. PMCHWT_multiple_scatterers,
  multiple_operator, AimAem, dualdef, GalA-MassP), preconditioners
  D, D^e, D^i, S^e, S^i (Section 3.1), right-hand side, restarted GMRES
  (Section 4), matvec counting (Table tab:matvecs) and the far field.
* ``mie``         Mie series of a dielectric sphere (Bohren & Huffman), the
  external pin of the whole solve.
* ``hmatrix``     the H-matrix model of Section 3.3: cluster trees, admissible
  blocks (disjoint boxes), ACA to a tolerance nu, the block-level cutoff chi
  (eq. nf_condition); ``pmchwt.PMCHWT(aca_P=(nu, chi))`` applies it to P.
* ``mixed``       the mixed (RWG, BC) discretisation of eq. mixed_discretisation:
  RWG rewritten on the barycentric mesh, cross blocks C(RWG, BC), C(BC, RWG).
* ``field``       the electric field at points off the surface from the
  Stratton–Chu representations (eqs. StrattonChu_int, StrattonChu_ext) with
  the potential operators of Section 2, for the |E|^2 plots of Section 5.

Where the paper is silent or garbled, the reading taken is stated in the
function that needs it.
"""
