// Library-internal access to a solver handle's device-resident solution
// (used by the landmark epilogue; not part of the public header).
#pragma once
#include "../../include/pinmpc.h"

namespace pinmpc {
// The trajectory of the last solve: xi [B][N][nx] on the handle's device.
// False when the handle has no solution yet.
bool solution_trajectory(const mpc_handle* h, const float** xi, int* B, int* N, int* nx, int* device);
}  // namespace pinmpc
