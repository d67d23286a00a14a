// Process-wide count of kernel launches made by this library (reported as evidence of which
// kernels ran inside a timed region).
#pragma once

namespace stmg {
void note_launch(int n = 1);
long long launch_count();
}  // namespace stmg
