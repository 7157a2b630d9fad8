// Host build of the 13-state model's device templates (csrc/quat_model.cuh):
// reads cases "dt x[13] u[4] lam[13] dir[17]" from stdin and prints, per case,
// the RK4 value F, the gradient of lam^T F with respect to (x, u), and, with
// dual numbers seeded in direction dir, the Jacobian-vector product dF and the
// Hessian-vector product of lam^T F.  The oracle comparison is in
// test_quat_model.py.
#include <cstdio>

#include "quat_model.cuh"

using bipm::Dual;

int main() {
  double dt;
  while (std::scanf("%lf", &dt) == 1) {
    double x[13], u[4], lam[13], dir[17];
    for (double& a : x) std::scanf("%lf", &a);
    for (double& a : u) std::scanf("%lf", &a);
    for (double& a : lam) std::scanf("%lf", &a);
    for (double& a : dir) std::scanf("%lf", &a);
    double F[13], F2[13], gx[13], gu[4];
    bipm::quat_rk4_value(x, u, dt, F);
    bipm::quat_rk4_fwd_rev(x, u, dt, lam, F2, gx, gu);
    Dual<double> xd[13], ud[4], Fd[13], gxd[13], gud[4];
    for (int i = 0; i < 13; ++i) xd[i] = Dual<double>{x[i], dir[i]};
    for (int i = 0; i < 4; ++i) ud[i] = Dual<double>{u[i], dir[13 + i]};
    bipm::quat_rk4_fwd_rev(xd, ud, dt, lam, Fd, gxd, gud);
    for (double a : F) std::printf("%.17g ", a);
    for (double a : F2) std::printf("%.17g ", a);
    for (double a : gx) std::printf("%.17g ", a);
    for (double a : gu) std::printf("%.17g ", a);
    for (auto& a : Fd) std::printf("%.17g ", a.d);
    for (auto& a : gxd) std::printf("%.17g ", a.d);
    for (auto& a : gud) std::printf("%.17g ", a.d);
    std::printf("\n");
  }
  return 0;
}
