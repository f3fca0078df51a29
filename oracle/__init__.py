"""CPU oracle for the RNS-CKKS hot path (TEST INFRASTRUCTURE ONLY).

Only tests/, the package smoke check and the benchmark's CPU-baseline leg may import this package.
The GPU library never imports, links or executes anything here.
"""
from .ckks import (  # noqa: F401
    CNNWeights, Ct, EncodedCNN, OracleCKKS, Pt, SwitchKey, cnn_bias_slots, cnn_encode, cnn_forward,
    cnn_galois_steps, cnn_mask_slots,
    cnn_plain, gen_primes, intt, is_prime, lib, min_psi, ntt, ntt_naive, philox4x64, power_products,
)
from .tensor import OracleTensor  # noqa: F401,E402
