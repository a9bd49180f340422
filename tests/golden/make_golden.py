"""Write the oracle's expected values for the full-size workloads.

Calls only the CPU oracle (``oracle/``) and the seeded generator
(``synth``).  For each workload it stores the length and SHA-256 of the
oracle's proof and the SHA-256 of the real outputs, so that GPU tests can
compare full-size proofs byte for byte without re-running the slow oracle.

    python tests/golden/make_golden.py medium slot
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


def main(names):
    o = Oracle()
    for name in names:
        circ = WORKLOADS[name]()
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
