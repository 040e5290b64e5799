// FP32 particle mode (positions, velocities, push and collisions in FP32;
// deposition in int64 fixed point; field solve and diagnostics in FP64).
#include "edupic_launch.cuh"

namespace edupic {
template struct Launch<float>;
}
