"""FP64 CPU oracle for the short-range PP path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import, call, link or execute anything in
this package.  The CUDA library and its Python binding never touch it, and it
shares no code with them.

Modules:
  force   -- the pair force of Eq. (split) summed directly over all sources
             (C, OpenMP, double precision) plus a numpy copy of the factor
  keys    -- Morton and Peano-Hilbert keys of the ground-grid + local octree
             ordering (Sec. 3.2, Sec. 4.1)
  tree    -- octree leaves, i-groups and the cutoff leaf-pair relation
  mlp     -- the 1-16-16-1 SiLU network that stands in for the factor:
             forward, backward and Adam in float64
  dtt     -- the tree part at the leaf level (opening criterion, leaf
             mass-centre bodies)
  pm      -- the long-range particle-mesh side (CIC, Green's function of
             the 3-point difference Laplacian with the split filter, central
             difference, CIC interpolation), numpy float64
  kdk     -- adaptive Kick-Drift-Kick block steps under the split force
             (Newtonian or flat Lambda-CDM drift/kick factors)
"""
