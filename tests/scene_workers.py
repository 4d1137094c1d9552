"""Worker-process helpers of the full-size multi-scene GPU tests (importable by spawned
processes): build one scene of a workload recipe with the library, and the oracle's digest of
its decoded values (SHA-256 of the fp32 bytes of the attributes and of the positions, so that
scenes of millions of Gaussians are compared bit for bit without shipping their arrays)."""
import hashlib

import numpy as np


def digests(attr: np.ndarray, pos: np.ndarray) -> tuple:
    return (hashlib.sha256(np.ascontiguousarray(attr, np.float32).tobytes()).hexdigest(),
            hashlib.sha256(np.ascontiguousarray(pos, np.float32).tobytes()).hexdigest())


def build_with_oracle(spec, train_steps):
    """(bitstream from the library, oracle digests of the scene's decoded values)."""
    from oracle import scene as S
    from paper_2607_12656_b300 import workloads
    from paper_2607_12656_b300.scenegen import fixed_bits, make_scene
    j, n, seed, depth, mode, lanes = spec
    sc = make_scene(n, seed)
    buf = workloads.encode_spec(spec, train_steps, scene=sc)
    P = S.prepare(sc.pos, sc.attr, depth, fixed_bits(seed) if mode == 0 else 8)
    return buf, digests(P.attr, P.pos)
