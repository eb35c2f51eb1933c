// Philox4x32-10 outputs of CURAND's device generator, for pinning the oracle's
// generator against an implementation it shares nothing with (test helper).
// stdin: "n" then n lines "seed subsequence offset"; stdout: one line of four
// words per request, curand4() of a state made by curand_init(seed,
// subsequence, offset).
#include <cstdio>
#include <vector>

#include <curand_kernel.h>

__global__ void k_curand4(const unsigned long long *req, uint4 *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(req[3 * i], req[3 * i + 1], req[3 * i + 2], &st);
    out[i] = curand4(&st);
}

int main()
{
    int n = 0;
    if (std::scanf("%d", &n) != 1 || n <= 0 || n > 1 << 20) return 2;
    std::vector<unsigned long long> req(3 * (size_t)n);
    for (int i = 0; i < 3 * n; ++i)
        if (std::scanf("%llu", &req[i]) != 1) return 2;
    unsigned long long *d_req = nullptr;
    uint4 *d_out = nullptr;
    if (cudaMalloc(&d_req, req.size() * sizeof(req[0])) != cudaSuccess) return 3;
    if (cudaMalloc(&d_out, (size_t)n * sizeof(uint4)) != cudaSuccess) return 3;
    cudaMemcpy(d_req, req.data(), req.size() * sizeof(req[0]), cudaMemcpyHostToDevice);
    k_curand4<<<(n + 127) / 128, 128>>>(d_req, d_out, n);
    std::vector<uint4> out(n);
    if (cudaMemcpy(out.data(), d_out, (size_t)n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess)
        return 4;
    for (int i = 0; i < n; ++i) std::printf("%u %u %u %u\n", out[i].x, out[i].y, out[i].z, out[i].w);
    cudaFree(d_req);
    cudaFree(d_out);
    return 0;
}
