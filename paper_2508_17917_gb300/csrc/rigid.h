// rigid.h -- one Newmark step of the 1-DOF oscillator (Eq. 1dof_oscillator,
// Algorithm 3), usable on the host and on the device.
#pragma once
#include <cuda_runtime.h>

namespace dg {

// Average-acceleration Newmark (beta = 1/4, gamma = 1/2) for
// M y'' + C y' + K y = F: the new acceleration solves the effective equation
// (M + dt C / 2 + dt^2 K / 4) a = F - C (y' + dt y''/2) - K (y + dt y' + dt^2 y''/4),
// then y and y' follow; vb = (y_new - y_old) / dt is the mesh velocity held
// over the next Runge-Kutta step.  Returns false (state untouched) when the
// effective mass vanishes or dt <= 0.
__host__ __device__ inline bool newmark_step(double M, double C, double K, double F, double dt, double &y,
                                             double &yd, double &ydd, double &vb)
{
    if (!(dt > 0.0)) return false;
    const double meff = M + 0.5 * dt * C + 0.25 * dt * dt * K;
    if (!(meff != 0.0)) return false;
    const double rhs = F - C * (yd + 0.5 * dt * ydd) - K * (y + dt * yd + 0.25 * dt * dt * ydd);
    const double a = rhs / meff;
    const double yn = y + dt * yd + 0.25 * dt * dt * (ydd + a);
    const double vn = yd + 0.5 * dt * (ydd + a);
    vb = (yn - y) / dt;
    y = yn;
    yd = vn;
    ydd = a;
    return true;
}

}  // namespace dg
