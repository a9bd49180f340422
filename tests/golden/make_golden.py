"""Write the oracle's expected values for the full-size workloads.

Calls only the CPU oracle (``oracle/``) and the seeded generator
(``synth``).  For each workload it stores the length and SHA-256 of the
oracle's proof and the SHA-256 of the real outputs, so that GPU tests can
compare full-size proofs byte for byte without re-running the slow oracle.

    python tests/golden/make_golden.py medium slot
    python tests/golden/make_golden.py batched:36 batched:31   # instances of the batched workload
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import Oracle  # noqa: E402

OUT = os.path.join(HERE, "oracle_full_size.json")
WORKLOADS = {"tiny": synth.tiny, "medium": synth.medium, "slot": synth.slot}


def _circuit(name: str):
    """A named workload, or instance j of the batched workload as "batched:j"
    (stored under "batched_j")."""
    if name.startswith("batched:"):
        j = int(name.split(":", 1)[1])
        return f"batched_{j}", synth.batched_instance(j)
    return name, WORKLOADS[name]()


def main(names):
    o = Oracle()
    o.set_threads(os.cpu_count() or 1)  # the proof bytes do not depend on it
    for arg in names:
        name, circ = _circuit(arg)
        t0 = time.time()
        x = synth.fr_bytes(synth.inputs_for(circ))
        outs = o.outputs(circ, x)
        proof = o.prove(circ, x)
        rec = {
            "workload": circ.name,
            "n_copies": circ.n_copies,
            "widths": [int(w) for w in circ.widths],
            "proof_len": len(proof),
            "proof_sha256": hashlib.sha256(proof).hexdigest(),
            "outputs_sha256": hashlib.sha256(outs).hexdigest(),
            "inputs_sha256": hashlib.sha256(x).hexdigest(),
            "oracle_seconds": round(time.time() - t0, 1),
        }
        # merge under a lock-free rename so parallel runs do not clobber
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[name] = rec
        tmp = OUT + f".tmp{os.getpid()}"
        json.dump(data, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, OUT)
        print(name, rec, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["tiny", "medium"])
