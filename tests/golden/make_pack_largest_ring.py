"""Writes pack_n65536_l5k2_n4.txt: the expected result of fast packing four
encrypted leaves at the largest ring (N = 2^16, 5 x 50-bit data primes, 2
special primes), computed by the CPU oracle alone (oracle.pack), for the GPU
parity test that cannot afford to run the oracle at this size itself (about
17 key switches of 42 schoolbook products of 2^16 points each).

Inputs, all seeded: secret key seed 61, rotation keys seed 62 (every d =
2^k + 1), four leaves encrypted in one call with seed 64 from messages drawn
with numpy's default_rng(63) in [-2^40, 2^40).  The file records the SHA-256
of the output residues (uint64 little-endian, [2][L][N] order) and a few
residues in clear.

    python tests/golden/make_pack_largest_ring.py
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

LOG_N, L, BITS, K = 16, 5, 50, 2
SK_SEED, RK_SEED, MSG_SEED, ENC_SEED, N_LEAVES = 61, 62, 63, 64, 4
OUT = os.path.join(HERE, "pack_n65536_l5k2_n4.txt")


def main():
    prm = O.make_params(LOG_N, L, BITS, K, BITS)
    s = O.keygen(prm, SK_SEED)
    keys = O.rotation_keys(prm, s, RK_SEED)
    msg = np.random.default_rng(MSG_SEED).integers(-2 ** 40, 2 ** 40, N_LEAVES * prm.n)
    cts = O.encrypt(prm, s, msg, ENC_SEED, N_LEAVES)
    out = O.pack(prm, keys, list(cts), n=N_LEAVES)
    digest = hashlib.sha256(np.ascontiguousarray(out, dtype="<u8").tobytes()).hexdigest()
    with open(OUT, "w") as f:
        f.write("# Fast packing of 4 encrypted leaves at N = 2^16, 5 x 50-bit + 2 special primes,\n")
        f.write("# written by tests/golden/make_pack_largest_ring.py (CPU oracle only).\n")
        f.write(f"# seeds: secret {SK_SEED}, rotation keys {RK_SEED}, messages {MSG_SEED}, encryption {ENC_SEED}\n")
        f.write(f"sha256 {digest}\n")
        for part in range(2):
            for limb in range(prm.L):
                f.write(f"residues {part} {limb} " + " ".join(str(int(v)) for v in out[part, limb, :4]) + "\n")
    print(OUT, digest)


if __name__ == "__main__":
    main()
