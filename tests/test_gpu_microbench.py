"""The microbenchmarks behind the rooflines of the back-projector and the
projector: shared-memory reads and FP32 fmas on every SM reach a good part
of the rates derived from the SM count and the maximum SM clock (2032 MHz on
the B300), and never exceed them (a rate above the derived peak would mean
the kernel does not do the work it reports)."""
import pytest
import torch

pytestmark = pytest.mark.gpu

SM_MAX_HZ = 2.032e9


@pytest.fixture(scope="module")
def P():
    import paper_1306_1392_b300 as P
    return P


def test_shared_memory_read_rate(P, cuda_device):
    sms = torch.cuda.get_device_properties(cuda_device).multi_processor_count
    derived = sms * 128 * SM_MAX_HZ                    # bytes/s: 128 B per clock and SM
    got = P.pyhst_microbench("smem_read", iters=4096, device=cuda_device)
    print(f"\nshared-memory reads {got / 1e12:.2f} TB/s = {got / derived:.3f} of {derived / 1e12:.2f}")
    assert 0.6 * derived < got <= 1.02 * derived


def test_fp32_fma_rate(P, cuda_device):
    sms = torch.cuda.get_device_properties(cuda_device).multi_processor_count
    derived = sms * 128 * 2 * SM_MAX_HZ                # flop/s: 128 fma lanes per clock and SM
    got = P.pyhst_microbench("fp32_fma", iters=4096, device=cuda_device)
    got2 = P.pyhst_microbench("fp32_fma2", iters=4096, device=cuda_device)
    print(f"\nfp32 fma {got / 1e12:.1f} TFLOP/s = {got / derived:.3f} of {derived / 1e12:.1f}; "
          f"paired {got2 / 1e12:.1f} TFLOP/s")
    assert 0.6 * derived < got <= 1.02 * derived
    assert got2 > 0.6 * derived


def test_mufu_rate(P, cuda_device):
    sms = torch.cuda.get_device_properties(cuda_device).multi_processor_count
    derived = sms * 16 * SM_MAX_HZ                     # MUFU operations/s: 16 per clock and SM
    got = P.pyhst_microbench("mufu", iters=2048, device=cuda_device)
    print(f"\nMUFU {got / 1e12:.2f} T ops/s = {got / derived:.3f} of {derived / 1e12:.2f}")
    assert 0.6 * derived < got <= 1.02 * derived
