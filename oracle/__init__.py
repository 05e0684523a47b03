"""FP64 CPU oracle for the streaming-collision LB scheme with the kinetic
diffuse-reflection wall (Meng & Zhang, arXiv:1209.5201).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg and reference arm (--impl reference) may import, call, link
or run anything in this package.  The
CUDA library never does, and this package never imports the library: the two
share no kernels, headers, helpers or table generators.  The oracle follows
the paper's push / ghost-layer description step by step in plain C (FP64,
no FMA contraction) and derives its own lattice tables in numpy.

Parity status per function (what pins it, see tests/test_oracle_pins.py):
  lattice.*                 pinned: Gaussian moment isotropy, closed forms
  orc_equilibrium           pinned: Maxwellian moments through the kept order
  orc_collide               pinned: exact conservation of rho, rho u (, energy);
                            its local tau through the viscosity law of the
                            bulk stress (mu = T and mu = T^0.7)
  orc_run (stream + wall)   pinned: free streaming by e_a (periodic in x),
                            re-emission from each ghost column by e_a,
                            specular return on the mirrored velocity,
                            rest / uniform-flow fixed points, per-step
                            zero net wall mass flux, slot bookkeeping,
                            positivity, Couette antisymmetry, NS slip limit
                            (Eq. (13)), NS temperature profile (Eq. (14), read
                            with U_w^2), second-order grid convergence
  orc_run_to_residual       pinned through the steady Couette profiles above
  orc_fluxes                pinned: sigma = q = 0 at equilibrium, traceless
                            thermal stress, Newtonian stress and Fourier heat
                            flux in the slow-shear bulk, uniform bulk shear
                            stress, energy balance q_y = -u_x sigma_xy under
                            grid refinement
"""
