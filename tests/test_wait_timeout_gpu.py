"""The bounded waits of the tensor-core kernels give up, on a GPU, without a
fault: a kernel compiled against the library's own wait helpers
(csrc/tc_ptx.cuh) waits on an mbarrier that nothing arrives at.

* mbar_wait returns false after the 2 s bound (not earlier, not much later);
* so does mbar_wait_or_abort_sleep, whose polls may sleep up to 1 us each;
* mbar_wait_or_abort and mbar_wait_or_abort_sleep return false at once when
  another role of the CTA has already set the abort flag;
* the context stays usable: a kernel launched afterwards runs normally.

The failing condition is made on purpose by never arriving, which is the
form of time-out test that leaves the GPU in a clean state (no trap, no
invalid access)."""
import os
import shutil
import subprocess
import tempfile

import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_10526_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "tc_ptx.cuh"
using namespace nk;

__global__ void k_wait(int *status, unsigned long long *elapsed) {
    __shared__ uint64_t bar;
    __shared__ volatile int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // phase 0 completes on one arrival, which never comes
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t0 = global_ns();
        status[0] = mbar_wait(&bar, 0) ? 1 : 0;
        elapsed[0] = global_ns() - t0;
        t0 = global_ns();
        status[2] = mbar_wait_or_abort_sleep(&bar, 0, &abort_flag) ? 1 : 0;
        elapsed[2] = global_ns() - t0;
        abort_flag = 1;  // another role gave up: the next waits return at once
        t0 = global_ns();
        status[1] = mbar_wait_or_abort(&bar, 0, &abort_flag) ? 1 : 0;
        elapsed[1] = global_ns() - t0;
        t0 = global_ns();
        status[3] = mbar_wait_or_abort_sleep(&bar, 0, &abort_flag) ? 1 : 0;
        elapsed[3] = global_ns() - t0;
    }
}

__global__ void k_after(int *x) { x[threadIdx.x] = (int)threadIdx.x + 1; }

int main() {
    int *status, *x;
    unsigned long long *elapsed;
    if (cudaMalloc(&status, 4 * sizeof(int)) || cudaMalloc(&elapsed, 4 * sizeof(unsigned long long)) ||
        cudaMalloc(&x, 32 * sizeof(int)))
        return 2;
    cudaMemset(status, 0xFF, 4 * sizeof(int));
    k_wait<<<1, 32>>>(status, elapsed);
    if (cudaDeviceSynchronize() != cudaSuccess) return 3;
    int hs[4];
    unsigned long long he[4];
    cudaMemcpy(hs, status, sizeof hs, cudaMemcpyDeviceToHost);
    cudaMemcpy(he, elapsed, sizeof he, cudaMemcpyDeviceToHost);
    k_after<<<1, 32>>>(x);
    int hx[32];
    const bool after_ok = cudaDeviceSynchronize() == cudaSuccess &&
                          cudaMemcpy(hx, x, sizeof hx, cudaMemcpyDeviceToHost) == cudaSuccess && hx[31] == 32;
    printf("%d %d %d %d %llu %llu %llu %llu %d\n", hs[0], hs[1], hs[2], hs[3], he[0], he[1], he[2], he[3],
           after_ok ? 1 : 0);
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc")
def test_bounded_mbarrier_wait_gives_up_and_the_context_survives():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "wait.cu")
        exe = os.path.join(d, "wait")
        with open(src, "w") as f:
            f.write(PROGRAM)
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-I", CSRC,
                        src, "-o", exe], check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stdout + r.stderr
        s0, s1, s2, s3, e0, e1, e2, e3, after = r.stdout.split()
    assert (int(s0), int(s1), int(s2), int(s3)) == (0, 0, 0, 0)  # every wait gave up
    assert 2.0e9 <= int(e0) < 4.0e9              # after the 2 s bound, not much later
    assert 2.0e9 <= int(e2) < 4.0e9              # the sleeping form keeps the same bound
    assert int(e1) < 5.0e7 and int(e3) < 5.0e7   # the abort flag ends both waits at once
    assert int(after) == 1                       # the context still runs kernels
