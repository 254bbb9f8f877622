"""optigpu for GB300: placeholder until the binding lands."""
