"""Small, fixed cases of the hot path for profiler captures.

Each case runs a reduced slice of the full 352-antenna workload a few times
(warm-up launches first), so that a capture of one kernel launch needs only a
few GB on the device:

    python -m paper_2606_04304_gb300.profile_cases imaging     # 256 channels, 256^2 images
    python -m paper_2606_04304_gb300.profile_cases detection   # 128^2 x 8192-channel cube
    python -m paper_2606_04304_gb300.profile_cases xengine     # 512 channels, K = 29
    python -m paper_2606_04304_gb300.profile_cases xengine299  # 128 channels, K = 299
    python -m paper_2606_04304_gb300.profile_cases upchan2400  # N = 2400, 704 inputs, 2 s
    python -m paper_2606_04304_gb300.profile_cases drift       # T = 8 x 512 channels x 128^2

Inputs are seeded and synthetic (the geometry of the full workload; random
visibilities / standardised cubes / spectra), generated on the device.
"""
from __future__ import annotations

import sys

import torch

import synth
from . import ovro


def imaging(repeats: int = 3) -> None:
    cfg = synth.make_config("full")
    pos = synth.antenna_positions(cfg)
    freqs = synth.fine_freqs_hz(cfg.nfft)[:256]
    g = torch.Generator(device="cuda").manual_seed(0)
    vis = torch.randint(-3000, 3000, (256, ovro.n_baselines(cfg.n_ant), 4, 2), generator=g, device="cuda",
                        dtype=torch.int32)
    for _ in range(repeats):
        ovro.grid_image(vis, pos, freqs, cfg.image_size, cfg.cell)


def detection(repeats: int = 2) -> None:
    g = torch.Generator(device="cuda").manual_seed(0)
    cube = torch.randn((8192, 128, 128), generator=g, device="cuda", dtype=torch.float32)
    freqs = synth.fine_freqs_hz([8192])
    for _ in range(repeats):
        ovro.detect(cube, 2.0 / 128, [8192], freqs)


def xengine(repeats: int = 3) -> None:
    n_ant, n_chan, k = 352, 512, 29
    g = torch.Generator(device="cuda").manual_seed(0)
    q = torch.randint(-127, 128, (n_chan * k * 2 * n_ant * 2,), generator=g, device="cuda",
                      dtype=torch.int16).to(torch.int8)
    for _ in range(repeats):
        ovro.correlate(q, n_ant, n_chan, k, ovro.XENG_TC)


def xengine299(repeats: int = 3) -> None:
    n_ant, n_chan, k = 352, 128, 299
    g = torch.Generator(device="cuda").manual_seed(0)
    q = torch.randint(-127, 128, (n_chan * k * 2 * n_ant * 2,), generator=g, device="cuda",
                      dtype=torch.int16).to(torch.int8)
    for _ in range(repeats):
        ovro.correlate(q, n_ant, n_chan, k, ovro.XENG_TC)


def upchan2400(repeats: int = 3) -> None:
    g = torch.Generator(device="cuda").manual_seed(0)
    volt = torch.randint(0, 256, (1, 48_000, 704), generator=g, device="cuda", dtype=torch.int32).to(torch.uint8)
    for _ in range(repeats):
        ovro.upchan(volt, [2400])


def drift(repeats: int = 2) -> None:
    g = torch.Generator(device="cuda").manual_seed(0)
    zsub = torch.randn((8, 512, 128, 128), generator=g, device="cuda", dtype=torch.float32)
    freqs = synth.fine_freqs_hz([512])
    for _ in range(repeats):
        ovro.drift_search(zsub, 2.0 / 128, [512], freqs, 12.0)


CASES = {"imaging": imaging, "detection": detection, "xengine": xengine, "xengine299": xengine299, "upchan2400": upchan2400,
         "drift": drift}


def main(argv) -> int:
    if len(argv) != 1 or argv[0] not in CASES:
        print(f"usage: python -m paper_2606_04304_gb300.profile_cases {{{','.join(CASES)}}}")
        return 2
    CASES[argv[0]]()
    torch.cuda.synchronize()
    print("ok", argv[0])
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
