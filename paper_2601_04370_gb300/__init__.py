"""GB300-native Monte Carlo polarization ray trace through a slab waveguide
with a partially reflective mirror array, its multilayer thin-film coatings
and the adjoint with respect to layer thicknesses (arXiv 2601.04370).

Modules:
  wg         - Python binding of libwg.so (the C ABI in include/wg.h)
  workloads  - seeded synthetic designs and trace configurations
  build      - builds libwg.so for sm_103a
The binding is imported on demand so that `workloads` needs no GPU library.
"""
