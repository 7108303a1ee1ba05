// Host driver for the kernels' Wilson interval (wilson_eq4 of
// paper_0912_2551_gb300/csrc/smc_device.cuh, compiled for the host through
// host_cuda_shims.h): reads lines "yes n z" and prints "p lo hi" (%.17g)
// for tests/test_wilson_device_host.py.
#include <stdio.h>

#include "host_cuda_shims.h"
#include "smc_device.cuh"

int main()
{
    unsigned long long yes, n;
    double z;
    while (scanf("%llu %llu %lf", &yes, &n, &z) == 3) {
        double out[3];
        wilson_eq4(yes, n, z, out);
        printf("%.17g %.17g %.17g\n", out[0], out[1], out[2]);
    }
    return 0;
}
