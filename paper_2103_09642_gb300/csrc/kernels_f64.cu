// FP64 particle mode.  Compiled with -fmad=false: every expression is
// evaluated with the roundings its source order implies.
#include "edupic_launch.cuh"

namespace edupic {
template struct Launch<double>;
}
