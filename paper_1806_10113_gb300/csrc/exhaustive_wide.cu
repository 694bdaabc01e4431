// exhaustive_wide.cu -- the exhaustive search's enumeration kernel in walk
// modes 6 to 8 (suffix constants in shared memory; tm_tuning.unroll), built
// as a translation unit of its own so that it compiles in parallel with
// exhaustive.cu, which holds the kernel's source and every other mode.
#define TM_ENUM_WIDE_MODES 1
#include "exhaustive.cu"
