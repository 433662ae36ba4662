// Collide kernel instantiations: double, 3D.
#define EF_T double
#define EF_D 3
#define EF_SUF f64_3d
#include "ef_collide_variant.inc"
